// Species-level connectivity (Fig. 1 lines 2-5, Sec. 2.1, Listing 2):
// XOR + popcount over every pair of determinants of one species, count ->
// scan -> fill with warp ballots, and the like-particle part of every
// Slater-Condon element evaluated once per species pair.
#include "problem.cuh"

namespace ci {

template <class T>
struct FilterArgs {
    int64_t n;
    int A, S, W;
    int mode;                  // ConnMode
    const uint64_t *bits;      // [n][W]
    const int32_t *twoM;       // [n]
    const int32_t *local;      // [n]
    const uint8_t *occ;        // [n][A]
    const T *eps, *U, *D, *C;  // like-particle tables of this species
    const int32_t *pair_row, *pair_col;
    const int32_t *tr_base;    // outer list: row offset of a proton move in the pn table
    const int32_t *tr_idx;     // neutron lists: column index of a neutron move
    const int32_t *q;          // [n] excess quanta
    const int64_t *p_row_base; // proton list: first basis row of every determinant
    int32_t *count;            // pass 0
    const int64_t *ptr;        // pass 1
    ConnEntry<T> *ent;         // pass 1
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

// Entry for row determinant s (bra) and partner t (ket).
template <class T>
__device__ __forceinline__ ConnEntry<T> make_entry_core(const FilterArgs<T> &a, int64_t s, int64_t t, const uint64_t *bs,
                                                        const uint64_t *bt, int d) {
    ConnEntry<T> e;
    e.tgt = (int32_t)t;
    e.local = a.local[t];
    const int S = a.S, W = a.W;
    if (d == 0) {
        // like-particle diagonal: one-body energies + every occupied pair
        const uint8_t *o = a.occ + s * a.A;
        T v = 0;
        for (int i = 0; i < a.A; ++i) v += a.eps[o[i]];
        for (int i = 0; i < a.A; ++i)
            for (int j = i + 1; j < a.A; ++j) v += a.D[o[i] * S + o[j]];
        e.info = make_info(0, 0, 0, 0);
        e.val = v;
        return e;
    }
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
        const T *u = a.U + ((int64_t)co * S + ao) * S;
        for (int i = 0; i < a.A; ++i)
            if (o[i] != ao) h += u[o[i]];
        e.info = make_info(1, par & 1, ao, co);
        if (a.mode == CONN_OUTER) e.local = a.tr_base[co * S + ao];
        else e.info |= (uint32_t)a.tr_idx[co * S + ao] << 17;
        e.val = h;
        return e;
    }
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
    T v = a.C[a.pair_row[c1 * S + d1] + a.pair_col[a1 * S + b1]];
    e.info = make_info(2, 0, a1, c1);
    e.val = (par & 1) ? -v : v;
    return e;
}

// Entry of row s, partner t; the proton list carries what the row kernels
// need about t (first basis row, q, change of 2M) instead of t itself.
template <class T>
__device__ __forceinline__ ConnEntry<T> make_entry(const FilterArgs<T> &a, int64_t s, int64_t t, const uint64_t *bs,
                                                   const uint64_t *bt, int d) {
    ConnEntry<T> e = make_entry_core<T>(a, s, t, bs, bt, d);
    if (a.mode == CONN_OUTER) {
        e.tgt = (int32_t)a.p_row_base[t];
        const int dslot = (a.twoM[t] - a.twoM[s]) / 2;
        e.info = (e.info & 0x1FFFFu) | ((uint32_t)a.q[t] << 17) | ((uint32_t)(dslot + 64) << 25);
    }
    return e;
}

// Each warp owns RW row determinants; the block's warps sweep the partner
// list in tiles of kTile determinants staged in shared memory (bits and 2M),
// so the list is read once per block.  Lanes take one partner each and a
// warp ballot per row keeps the partners in ascending order.
constexpr int kTile = 512;

template <class T, int W, int RW>
__global__ void __launch_bounds__(256) k_filter(const FilterArgs<T> *jobs, const int64_t *job_blk, int njobs,
                                                int pass) {
    __shared__ uint64_t sbits[kTile * W];
    __shared__ int32_t sm2[kTile];
    int lo = 0, hi = njobs - 1;  // the job (one list of one problem) of this block
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (job_blk[mid] <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const FilterArgs<T> a = jobs[lo];  // by value: stores to ent cannot alias it
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t row0 = (((int64_t)blockIdx.x - job_blk[lo]) * 8 + wid) * RW;
    uint64_t bs[RW][kMaxWords];
    int ms[RW];
    int64_t out[RW];
    int cnt[RW];
#pragma unroll
    for (int i = 0; i < RW; ++i) {
        const int64_t s = row0 + i;
        const bool ok = s < a.n;
#pragma unroll
        for (int w = 0; w < kMaxWords; ++w) bs[i][w] = (ok && w < W) ? a.bits[s * W + w] : 0ull;
        ms[i] = ok ? a.twoM[s] : 0;
        out[i] = (ok && pass) ? a.ptr[s] : 0;
        cnt[i] = 0;
    }
    for (int64_t t0 = 0; t0 < a.n; t0 += kTile) {
        const int nt = (int)min((int64_t)kTile, a.n - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt * W; e += blockDim.x) sbits[e] = a.bits[t0 * W + e];
        for (int e = threadIdx.x; e < nt; e += blockDim.x) sm2[e] = a.twoM[t0 + e];
        __syncthreads();
        for (int c0 = 0; c0 < nt; c0 += 32) {
            const int tl = c0 + lane;
            const bool tv = tl < nt;
            uint64_t bt[kMaxWords] = {0ull, 0ull};
#pragma unroll
            for (int w = 0; w < W; ++w) bt[w] = tv ? sbits[tl * W + w] : 0ull;
            const int mt = tv ? sm2[tl] : 0;
#pragma unroll
            for (int i = 0; i < RW; ++i) {
                int d = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) d += __popcll(bs[i][w] ^ bt[w]);
                const bool sameM = mt == ms[i];
                bool keep;
                if (a.mode == CONN_OUTER) keep = d <= 2 || (d == 4 && sameM);
                else if (a.mode == CONN_L2) keep = d <= 2;
                else keep = d <= 4 && sameM;
                keep = keep && tv && (row0 + i < a.n);
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (pass && keep) {
                    const int rank = __popc(bal & ((1u << lane) - 1u));
                    a.ent[out[i] + rank] = make_entry<T>(a, row0 + i, t0 + tl, bs[i], bt, d);
                    a.tgt[out[i] + rank] = (int32_t)(t0 + tl);
                }
                out[i] += __popc(bal);
                cnt[i] += __popc(bal);
            }
        }
    }
    if (!pass && lane == 0) {
#pragma unroll
        for (int i = 0; i < RW; ++i)
            if (row0 + i < a.n) a.count[row0 + i] = cnt[i];
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
    launch("k_filter", k_filter<T, W, RW>, (unsigned)blk.back(), 256, 0, s, (const FilterArgs<T> *)dj.ptr,
           (const int64_t *)db.ptr, (int)jobs.size(), pass);
}

template <class T>
static void filter_pass(const std::vector<FilterArgs<T>> &jobs, int pass, cudaStream_t s) {
    // rows per warp: 4 only when that still leaves every SM 16 blocks of
    // 8 warps (the sweep is latency bound, so more warps beat more reuse)
    std::vector<FilterArgs<T>> j1, j2;
    int64_t rows = 0;
    for (auto &j : jobs) {
        (j.W == 1 ? j1 : j2).push_back(j);
        rows += j.n;
    }
    const bool wide = rows >= (int64_t)sm_count() * 16 * 32;
    if (wide) { launch_filter<T, 1, 4>(j1, pass, s); launch_filter<T, 2, 4>(j2, pass, s); }
    else { launch_filter<T, 1, 1>(j1, pass, s); launch_filter<T, 2, 1>(j2, pass, s); }
}

// Segment tables of one problem's neutron lists.
//   seg2[n][ds][c]: end (relative to ptr[n]) of the L2 entries whose key
//   (2M, q) is <= (2M_n + 2(ds-K), c); with no Nmax cut the q part is ignored.
//   seg4[n][c]: end (relative) of the L4 entries with q <= c (all same 2M).
template <class T>
struct SegJob {
    int64_t n;
    int nds, nq, K, cut;
    const int64_t *p2, *p4;
    const ConnEntry<T> *e2, *e4;
    const int32_t *twoM, *q;
    int32_t *seg2, *seg4;
};

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
        const int64_t n2 = j.n * j.nds * j.nq;
        if (r < n2) {
            const int c = (int)(r % j.nq);
            const int ds = (int)((r / j.nq) % j.nds);
            const int64_t s = r / ((int64_t)j.nq * j.nds);
            const int mt = j.twoM[s] + 2 * (ds - j.K);
            int64_t lo = j.p2[s], hi = j.p2[s + 1];  // first entry with key > (mt, c)
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int tg = j.e2[mid].tgt;
                const int mm = j.twoM[tg];
                const bool le = mm < mt || (mm == mt && (!j.cut || j.q[tg] <= c));
                if (le) lo = mid + 1; else hi = mid;
            }
            j.seg2[r] = (int32_t)(lo - j.p2[s]);
        } else {
            r -= n2;
            const int c = (int)(r % j.nq);
            const int64_t s = r / j.nq;
            int64_t lo = j.p4[s], hi = j.p4[s + 1];
            if (j.cut) {
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (j.q[j.e4[mid].tgt] <= c) lo = mid + 1; else hi = mid;
                }
            } else {
                lo = hi;
            }
            j.seg4[r] = (int32_t)(lo - j.p4[s]);
        }
    }
}

template <class T>
static FilterArgs<T> filter_job(Problem *p, int species, int mode) {
    SpeciesList &sp = p->sp[species];
    Tables<T> &t = p->tables<T>();
    FilterArgs<T> a{};
    a.n = sp.n; a.A = sp.A; a.S = p->S; a.W = sp.W; a.mode = mode;
    a.bits = sp.d_bits.ptr; a.twoM = sp.d_twoM.ptr; a.local = sp.d_local.ptr; a.occ = sp.d_occ.ptr;
    a.q = sp.d_q.ptr;
    a.p_row_base = species == 0 ? p->d_p_row_base.ptr : nullptr;
    a.eps = t.eps.ptr;
    a.U = species == 0 ? t.Upp.ptr : t.Unn.ptr;
    a.D = species == 0 ? t.Dpp.ptr : t.Dnn.ptr;
    a.C = species == 0 ? t.Cpp.ptr : t.Cnn.ptr;
    a.pair_row = p->like_row.ptr; a.pair_col = p->like_col.ptr;
    a.tr_base = p->tr_base.ptr; a.tr_idx = p->tr_idx.ptr;
    return a;
}

// Species connectivity of every problem of ps (Fig. 1 lines 2-5): count
// pass, one scan over all lists, one allocation, fill pass, segment tables.
template <class T>
void species_filter_group(const std::vector<Problem *> &ps_in, cudaStream_t s) {
    std::vector<Problem *> ps;
    for (Problem *p : ps_in)
        if (!p->conn<T>().ready) ps.push_back(p);
    if (ps.empty()) return;
    for (Problem *p : ps) enumerate_basis(p, s);
    stage_tables_group<T>(ps, s);
    // jobs: 3 lists per problem, their counts side by side in one array
    std::vector<FilterArgs<T>> jobs;
    std::vector<ConnList<T> *> lists;
    std::vector<int64_t> cnt_off(1, 0);
    for (Problem *p : ps) {
        Connectivity<T> &c = p->conn<T>();
        const int modes[3] = {CONN_OUTER, CONN_L2, CONN_L4};
        ConnList<T> *ls[3] = {&c.outer, &c.l2, &c.l4};
        for (int i = 0; i < 3; ++i) {
            jobs.push_back(filter_job<T>(p, i == 0 ? 0 : 1, modes[i]));
            lists.push_back(ls[i]);
            cnt_off.push_back(cnt_off.back() + jobs.back().n);
        }
    }
    const int64_t ncnt = cnt_off.back();
    DevBuf<int32_t> cnt((size_t)ncnt);
    auto offs = std::make_shared<DevBuf<int64_t>>((size_t)ncnt + 1);
    for (size_t i = 0; i < jobs.size(); ++i) jobs[i].count = cnt.ptr + cnt_off[i];
    filter_pass<T>(jobs, 0, s);
    exclusive_scan_i32(cnt.ptr, ncnt, offs->ptr, ps[0]->scan_scratch, s);
    // list boundaries: hb[i] = offs[cnt_off[i]]
    std::vector<int64_t> hb = gather_i64(offs->ptr, cnt_off, s);
    auto ents = std::make_shared<DevBuf<ConnEntry<T>>>((size_t)hb.back());
    auto tgts = std::make_shared<DevBuf<int32_t>>((size_t)hb.back());
    for (size_t i = 0; i < jobs.size(); ++i) {
        ConnList<T> &L = *lists[i];
        L.ptr_buf = offs;
        L.ent_buf = ents;
        L.tgt_buf = tgts;
        L.tgt = tgts->ptr;
        L.ptr = offs->ptr + cnt_off[i];
        L.ent = ents->ptr;
        L.n = jobs[i].n;
        L.first = hb[i];
        L.total = hb[i + 1] - hb[i];
        jobs[i].ptr = L.ptr;
        jobs[i].ent = L.ent;
        jobs[i].tgt = tgts->ptr;
    }
    filter_pass<T>(jobs, 1, s);
    // segment tables of the neutron lists
    std::vector<SegJob<T>> sj;
    std::vector<int64_t> soff(1, 0);
    for (Problem *p : ps) {
        Connectivity<T> &c = p->conn<T>();
        SpeciesList &Nn = p->sp[1];
        c.seg2.alloc((size_t)Nn.n * p->nds * Nn.nq);
        c.seg4.alloc((size_t)Nn.n * Nn.nq);
        SegJob<T> j{};
        j.n = Nn.n; j.nds = p->nds; j.nq = Nn.nq; j.K = p->K; j.cut = p->nmax >= 0;
        j.p2 = c.l2.ptr; j.p4 = c.l4.ptr; j.e2 = c.l2.ent; j.e4 = c.l4.ent;
        j.twoM = Nn.d_twoM.ptr; j.q = Nn.d_q.ptr; j.seg2 = c.seg2.ptr; j.seg4 = c.seg4.ptr;
        const int64_t w = Nn.n * p->nds * Nn.nq + Nn.n * Nn.nq;
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
    for (Problem *p : ps) p->conn<T>().ready = true;
}

template void species_filter_group<float>(const std::vector<Problem *> &, cudaStream_t);
template void species_filter_group<double>(const std::vector<Problem *> &, cudaStream_t);


}  // namespace ci
