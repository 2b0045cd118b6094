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
    int32_t *count;            // pass 0
    const int64_t *ptr;        // pass 1
    ConnEntry<T> *ent;         // pass 1
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
__device__ ConnEntry<T> make_entry(const FilterArgs<T> &a, int64_t s, int64_t t, const uint64_t *bs,
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

// Each warp owns RW row determinants; the block's warps sweep the partner
// list in tiles of kTile determinants staged in shared memory (bits and 2M),
// so the list is read once per block.  Lanes take one partner each and a
// warp ballot per row keeps the partners in ascending order.
constexpr int kTile = 512;

template <class T, int W, int RW>
__global__ void __launch_bounds__(256) k_filter(FilterArgs<T> a, int pass) {
    __shared__ uint64_t sbits[kTile * W];
    __shared__ int32_t sm2[kTile];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t row0 = ((int64_t)blockIdx.x * 8 + wid) * RW;
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

template <class T, int W>
static void launch_filter(const FilterArgs<T> &a, int pass, cudaStream_t s) {
    // rows per warp: 4 when that still gives every SM a few blocks
    if (a.n >= (int64_t)sm_count() * 4 * 32) {
        launch("k_filter", k_filter<T, W, 4>, (unsigned)((a.n + 31) / 32), 256, 0, s, a, pass);
    } else {
        launch("k_filter", k_filter<T, W, 1>, (unsigned)((a.n + 7) / 8), 256, 0, s, a, pass);
    }
}

// seg2[n][ds][c]: end (relative to ptr[n]) of the L2 entries whose key
// (2M, q) is <= (2M_n + 2(ds-K), c); with no Nmax cut the q part is ignored.
__global__ void k_seg2(int64_t n, int nds, int nq, int K, int cut, const int64_t *ptr,
                       const ConnEntry<float> *ent_f, const ConnEntry<double> *ent_d,
                       const int32_t *twoM, const int32_t *q, int32_t *seg) {
    int64_t total = n * nds * nq;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(e % nq);
        int ds = (int)((e / nq) % nds);
        int64_t s = e / ((int64_t)nq * nds);
        int mt = twoM[s] + 2 * (ds - K);
        int64_t lo = ptr[s], hi = ptr[s + 1];  // first entry with key > (mt, c)
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            int tg = ent_f ? ent_f[mid].tgt : ent_d[mid].tgt;
            int mm = twoM[tg];
            bool le = mm < mt || (mm == mt && (!cut || q[tg] <= c));
            if (le) lo = mid + 1; else hi = mid;
        }
        seg[e] = (int32_t)(lo - ptr[s]);
    }
}

// seg4[n][c]: end (relative) of the L4 entries with q <= c (all same 2M).
__global__ void k_seg4(int64_t n, int nq, int cut, const int64_t *ptr, const ConnEntry<float> *ent_f,
                       const ConnEntry<double> *ent_d, const int32_t *q, int32_t *seg) {
    int64_t total = n * nq;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(e % nq);
        int64_t s = e / nq;
        int64_t lo = ptr[s], hi = ptr[s + 1];
        if (cut) {
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                int tg = ent_f ? ent_f[mid].tgt : ent_d[mid].tgt;
                if (q[tg] <= c) lo = mid + 1; else hi = mid;
            }
        } else {
            lo = hi;
        }
        seg[e] = (int32_t)(lo - ptr[s]);
    }
}

template <class T>
static void build_list(Problem *p, int species, int mode, ConnList<T> &L, cudaStream_t s) {
    SpeciesList &sp = p->sp[species];
    Tables<T> &t = p->tables<T>();
    FilterArgs<T> a;
    a.n = sp.n; a.A = sp.A; a.S = p->S; a.W = sp.W; a.mode = mode;
    a.bits = sp.d_bits.ptr; a.twoM = sp.d_twoM.ptr; a.local = sp.d_local.ptr; a.occ = sp.d_occ.ptr;
    a.eps = t.eps.ptr;
    a.U = species == 0 ? t.Upp.ptr : t.Unn.ptr;
    a.D = species == 0 ? t.Dpp.ptr : t.Dnn.ptr;
    a.C = species == 0 ? t.Cpp.ptr : t.Cnn.ptr;
    a.pair_row = p->like_row.ptr; a.pair_col = p->like_col.ptr;
    a.tr_base = p->tr_base.ptr; a.tr_idx = p->tr_idx.ptr;
    DevBuf<int32_t> cnt(sp.n);
    a.count = cnt.ptr; a.ptr = nullptr; a.ent = nullptr;
    L.ptr.alloc(sp.n + 1);
    if (sp.n == 0) {
        CI_CUDA(cudaMemsetAsync(L.ptr.ptr, 0, sizeof(int64_t), s));
        L.total = 0;
        L.ent.alloc(1);
        return;
    }
    if (sp.W == 1) launch_filter<T, 1>(a, 0, s);
    else launch_filter<T, 2>(a, 0, s);
    CI_CHECK_LAUNCH();
    exclusive_scan_i32(cnt.ptr, sp.n, L.ptr.ptr, p->scan_scratch, s);
    CI_CUDA(cudaMemcpyAsync(&L.total, L.ptr.ptr + sp.n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CI_CUDA(cudaStreamSynchronize(s));
    L.ent.alloc(L.total);
    a.ptr = L.ptr.ptr; a.ent = L.ent.ptr;
    if (sp.W == 1) launch_filter<T, 1>(a, 1, s);
    else launch_filter<T, 2>(a, 1, s);
    CI_CHECK_LAUNCH();
}

template <class T>
void species_filter(Problem *p, cudaStream_t s) {
    Connectivity<T> &c = p->conn<T>();
    if (c.ready) return;
    stage_tables<T>(p, s);
    build_list<T>(p, 0, CONN_OUTER, c.outer, s);
    build_list<T>(p, 1, CONN_L2, c.l2, s);
    build_list<T>(p, 1, CONN_L4, c.l4, s);
    SpeciesList &Nn = p->sp[1];
    const int cut = p->nmax >= 0;
    c.seg2.alloc((size_t)Nn.n * p->nds * Nn.nq);
    c.seg4.alloc((size_t)Nn.n * Nn.nq);
    if (Nn.n > 0) {
        const bool f = sizeof(T) == 4;
        launch("k_seg2", k_seg2, grid_for(Nn.n * p->nds * Nn.nq, 256), 256, 0, s, 
            Nn.n, p->nds, Nn.nq, p->K, cut, c.l2.ptr.ptr,
            f ? (const ConnEntry<float> *)c.l2.ent.ptr : nullptr,
            f ? nullptr : (const ConnEntry<double> *)c.l2.ent.ptr, Nn.d_twoM.ptr, Nn.d_q.ptr, c.seg2.ptr);
        launch("k_seg4", k_seg4, grid_for(Nn.n * Nn.nq, 256), 256, 0, s, 
            Nn.n, Nn.nq, cut, c.l4.ptr.ptr, f ? (const ConnEntry<float> *)c.l4.ent.ptr : nullptr,
            f ? nullptr : (const ConnEntry<double> *)c.l4.ent.ptr, Nn.d_q.ptr, c.seg4.ptr);
        CI_CHECK_LAUNCH();
    }
    CI_CUDA(cudaStreamSynchronize(s));
    c.ready = true;
}

template void species_filter<float>(Problem *, cudaStream_t);
template void species_filter<double>(Problem *, cudaStream_t);

}  // namespace ci
