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

// One warp per row determinant s; lanes sweep the partners t in order.
template <class T, int W>
__global__ void __launch_bounds__(256) k_filter(FilterArgs<T> a, int pass) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < a.n; s += nwarps) {
        uint64_t bs[kMaxWords] = {0, 0};
        for (int w = 0; w < W; ++w) bs[w] = a.bits[s * W + w];
        const int ms = a.twoM[s];
        int64_t out = pass ? a.ptr[s] : 0;
        int cnt = 0;
        for (int64_t base = 0; base < a.n; base += 32) {
            int64_t t = base + lane;
            bool keep = false;
            int d = 0;
            uint64_t bt[kMaxWords] = {0, 0};
            if (t < a.n) {
                for (int w = 0; w < W; ++w) {
                    bt[w] = a.bits[t * W + w];
                    d += __popcll(bs[w] ^ bt[w]);
                }
                bool sameM = a.twoM[t] == ms;
                if (a.mode == CONN_OUTER) keep = d <= 2 || (d == 4 && sameM);
                else if (a.mode == CONN_L2) keep = d <= 2;
                else keep = d <= 4 && sameM;
            }
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (pass && keep) {
                int rank = __popc(bal & ((1u << lane) - 1u));
                a.ent[out + rank] = make_entry<T>(a, s, t, bs, bt, d);
            }
            out += __popc(bal);
            cnt += __popc(bal);
        }
        if (!pass && lane == 0) a.count[s] = cnt;
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
    DevBuf<int32_t> cnt(sp.n);
    a.count = cnt.ptr; a.ptr = nullptr; a.ent = nullptr;
    L.ptr.alloc(sp.n + 1);
    if (sp.n == 0) {
        CI_CUDA(cudaMemsetAsync(L.ptr.ptr, 0, sizeof(int64_t), s));
        L.total = 0;
        L.ent.alloc(1);
        return;
    }
    const int thr = 256;
    int grid = grid_for(sp.n * 32, thr, sm_count() * 8);
    if (sp.W == 1) launch("k_filter", k_filter<T, 1>, grid, thr, 0, s, a, 0);
    else launch("k_filter", k_filter<T, 2>, grid, thr, 0, s, a, 0);
    CI_CHECK_LAUNCH();
    exclusive_scan_i32(cnt.ptr, sp.n, L.ptr.ptr, p->scan_scratch, s);
    CI_CUDA(cudaMemcpyAsync(&L.total, L.ptr.ptr + sp.n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CI_CUDA(cudaStreamSynchronize(s));
    L.ent.alloc(L.total);
    a.ptr = L.ptr.ptr; a.ent = L.ent.ptr;
    if (sp.W == 1) launch("k_filter", k_filter<T, 1>, grid, thr, 0, s, a, 1);
    else launch("k_filter", k_filter<T, 2>, grid, thr, 0, s, a, 1);
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
