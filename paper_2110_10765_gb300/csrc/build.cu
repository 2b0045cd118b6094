// Count -> scan -> fill of the Hamiltonian rows (Fig. 1, count and fill,
// Sec. 2.2-2.3).  One warp owns one row (p, n).  The row's partners are
// the proton partners p' of p (ascending) crossed with segments of the
// neutron lists of n: for p' two states away (list O2), the L2(n) entries
// in the 2M block that pairs with p' and within the Nmax cut; for p' = p,
// the L4(n) entries; for p' four states away (list O4, same 2M), n itself.
// Only partners that can still meet a neutron partner under the cut are
// visited: per 2M slot of O2 the q-prefix up to Nmax - (smallest q of the
// matching L2 slot), and the q-prefix of O4 up to Nmax - q(n).  The O4
// partners interleave with the same-2M slot of O2 by column.  Columns
// therefore come out ascending without sorting, and every lane writes its
// own slot of a coalesced run (the deterministic counterpart of Listing 7's
// atomic capture).
#include <climits>

#include <cuda_bf16.h>

#include "problem.cuh"

namespace ci {

template <class T>
struct RowArgs {
    int64_t dim;
    int S, W, nq, nds, K, nmax, twoM;
    const int32_t *row_p, *row_n;
    const int64_t *p_row_base;
    const int32_t *p_q, *p_twoM, *n_q, *n_twoM, *n_local;
    const uint64_t *p_bits, *n_bits;
    const int64_t *o_ptr, *o4_ptr, *l2_ptr, *l4_ptr;
    const ConnEntry<T> *o_ent, *o4_ent, *l2_ent, *l4_ent;
    const int32_t *o_xr;       // cross ranks of the same-2M proton entries (O2 <-> O4)
    const int32_t *seg2, *seg4, *qmin2, *oseg2, *oseg4;
    const T *Upn, *Wpn, *Dpn, *Tpn;
    int32_t *row_cnt;          // count pass
    const int64_t *row_ptr;    // fill pass
    int32_t *col;
    T *val;
};

// Segment of neutron partners that the proton partner entry e opens for
// row (p, n).  kind 0: n itself (one entry); 1: L2(n)[beg, beg+len);
// 2: L4(n)[0, len).
template <class T>
__device__ __forceinline__ void partner_segment(const RowArgs<T> &a, int p, int n, const ConnEntry<T> &e,
                                                int &kind, int &beg, int &len) {
    const int dc = info_dcode(e.info);
    const int qp = info_q(e.info);   // q of the proton partner
    kind = 0; beg = 0; len = 0;
    if (dc == 2) {  // four states moved among protons: the neutrons stay put
        if (a.nmax < 0 || qp + a.n_q[n] <= a.nmax) len = 1;
        return;
    }
    int c = 0;
    if (a.nmax >= 0) {
        c = a.nmax - qp;
        if (c < 0) return;
        if (c > a.nq - 1) c = a.nq - 1;
    }
    if (dc == 0) {  // p' = p: every same-2M neutron partner of n
        kind = 2;
        len = a.seg4[(int64_t)n * a.nq + c];
        return;
    }
    kind = 1;       // one proton moved: neutron partners at most one move away
    // target 2M of n' is twoM - 2M(p') = 2M(n) - (2M(p') - 2M(p))
    const int ds = a.K - info_dslot(e.info);
    if (ds < 0 || ds >= a.nds) return;
    const int32_t *sg = a.seg2 + (int64_t)n * a.nds * a.nq;
    beg = ds == 0 ? 0 : sg[(ds - 1) * a.nq + (a.nq - 1)];
    int end = sg[ds * a.nq + c];
    len = end > beg ? end - beg : 0;
}

__device__ __forceinline__ int warp_incl_scan_i32(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// problem of global row gr in a group (row_off: [G+1])
__device__ __forceinline__ int group_of(const int64_t *row_off, int G, int64_t gr) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= gr) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Admissible O2 partners of row (p, n) in 2M slots [g_lo, g_hi), ascending,
// 32 at a time: body(e, valid) with e the lane's entry of the O2 list.
// Warp-uniform calls.
template <class T, class F>
__device__ __forceinline__ void for_o2(const RowArgs<T> &a, int p, int n, int g_lo, int g_hi, F &&body) {
    const int lane = threadIdx.x & 31;
    const int64_t e0 = a.o_ptr[p];
    const int32_t *os = a.oseg2 + (int64_t)p * a.nds * a.nq;
    const int32_t *qm = a.qmin2 + (int64_t)n * a.nds;
    for (int g0 = g_lo; g0 < g_hi; g0 += 32) {
        const int g = g0 + lane;
        int gb = 0, gl = 0;
        if (g < g_hi) {
            gb = g == 0 ? 0 : os[(g - 1) * a.nq + a.nq - 1];
            int ge;
            if (a.nmax < 0) {
                ge = os[g * a.nq + a.nq - 1];
            } else {
                // partners p' of slot g meet the L2(n) slot 2K - g; they need
                // q(p') <= Nmax - (smallest q there)
                int c = a.nmax - qm[2 * a.K - g];
                if (c > a.nq - 1) c = a.nq - 1;
                ge = c < 0 ? gb : os[g * a.nq + c];
            }
            gl = ge > gb ? ge - gb : 0;
        }
        const int incl = warp_incl_scan_i32(gl);
        const int excl = incl - gl;
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        for (int t0 = 0; t0 < tot; t0 += 32) {
            const int t = t0 + lane;
            int j = 0;  // last slot starting at or before t
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int v = __shfl_sync(0xffffffffu, excl, j + step);
                if (v <= t) j += step;
            }
            const int64_t e = e0 + __shfl_sync(0xffffffffu, gb, j) + (t - __shfl_sync(0xffffffffu, excl, j));
            body(e, t < tot);
        }
    }
}

// Admissible O4 partners of row (p, n): the q-prefix up to Nmax - q(n).
template <class T>
__device__ __forceinline__ int o4_count(const RowArgs<T> &a, int p, int n) {
    const int64_t b = a.o4_ptr[p];
    if (a.nmax < 0) return (int)(a.o4_ptr[p + 1] - b);
    int c = a.nmax - a.n_q[n];
    if (c < 0) return 0;
    if (c > a.nq - 1) c = a.nq - 1;
    return a.oseg4[(int64_t)p * a.nq + c];
}

template <class T>
__global__ void __launch_bounds__(256) k_count_rows(const RowArgs<T> *args, const int64_t *row_off, int G) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t rows = row_off[G];
    for (int64_t gr = warp; gr < rows; gr += nwarps) {
        const int g = group_of(row_off, G, gr);
        const RowArgs<T> &a = args[g];
        const int64_t r = gr - row_off[g];
        const int p = a.row_p[r], n = a.row_n[r];
        int cnt = 0;
        for_o2<T>(a, p, n, 0, a.nds, [&](int64_t e, bool ok) {
            if (ok) {
                int kind, beg, len;
                partner_segment<T>(a, p, n, a.o_ent[e], kind, beg, len);
                cnt += len;
            }
        });
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) a.row_cnt[r] = cnt + o4_count<T>(a, p, n);
    }
}

// sum over the occupied states k of determinant s (W-word bit strings) of
// tab[k], in ascending k.  For S <= 128 the states are taken four at a time
// and their four loads issued before the adds (the same order of adds).
template <class T>
__device__ __forceinline__ T sum_over_bits(const T *tab, const uint64_t *bits, int s, int W) {
    const uint64_t *b = bits + (int64_t)s * W;
    T sum = 0;
    if (W <= 2) {   // S <= 128: both words loaded up front, no loop over words
        uint64_t w0 = b[0], w1 = W > 1 ? b[1] : 0ull;
        while (w0 | w1) {
            int k[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (w0) {
                    k[u] = __ffsll((long long)w0) - 1;
                    w0 &= w0 - 1;
                } else if (w1) {
                    k[u] = 64 + __ffsll((long long)w1) - 1;
                    w1 &= w1 - 1;
                } else {
                    k[u] = -1;
                }
            }
            T x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = k[u] >= 0 ? tab[k[u]] : (T)0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k[u] >= 0) sum += x[u];
        }
        return sum;
    }
    for (int w = 0; w < W; ++w) {
        uint64_t x = b[w];
        while (x) { const int k = __ffsll((long long)x) - 1; x &= x - 1; sum += tab[64 * w + k]; }
    }
    return sum;
}

// Row context of the fill.  The bit strings of p and n are only needed by
// the rare spectator sums and are loaded there.
struct RowCtx {
    int p, n, n_local;
    int64_t l2b, l4b;
};

// One chunk of up to 32 O2 partners (one per lane: entry ep, segment kind,
// beg, len; extra = elements of other partners placed before this one's
// segment).  The lane's segment goes to out + (exclusive scan of len) +
// extra, written in three phases without sorting:
//   0. four protons moved: one element (n' = n), by its lane;
//   1. one proton moved: the segments of L2(n) are expanded with the warp's
//      lanes balanced over the elements (a search over segment starts);
//   2. p' = p: the warp walks the row's L4(n) segment contiguously.
// Returns the chunk's element count.
template <class T, class Emit>
__device__ __forceinline__ int fill_chunk(const RowArgs<T> &a, const RowCtx &x, const ConnEntry<T> &ep, int kind,
                                          int beg, int len, int extra, int64_t out, Emit &em) {
    const int lane = threadIdx.x & 31;
    const int S = a.S;
    const int incl = warp_incl_scan_i32(len);
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int64_t pos = out + (incl - len) + extra;
    const int colbase = ep.tgt;   // first basis row of the proton partner
    // 0. four protons moved: the neutrons stay, one element
    if (kind == 0 && len == 1) em.put(a, pos, colbase + x.n_local, ep.val);
    // (2,0) elements below (one proton moved, the neutrons spectators) take a
    // value that depends on the partner alone: its lane forms it here, once
    T hspec = 0;
    if (kind == 1 && len > 0 && info_dslot(ep.info) == 0) {
        const T *u = a.Upn + ((int64_t)info_c(ep.info) * S + info_a(ep.info)) * S;
        hspec = ep.val + sum_over_bits<T>(u, a.n_bits, x.n, a.W);
    }
    // 1. one proton moved (a -> c): L2(n)[beg, beg+len)
    const int len1 = kind == 1 ? len : 0;
    const int incl1 = warp_incl_scan_i32(len1);
    const int excl1 = incl1 - len1;
    const int total1 = __shfl_sync(0xffffffffu, incl1, 31);
    for (int t0 = 0; t0 < total1; t0 += 32) {
        const int t = t0 + lane;
        int j = 0;  // last lane whose kind-1 segment starts at or before t
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, excl1, j + step);
            if (v <= t) j += step;
        }
        const int k = t - __shfl_sync(0xffffffffu, excl1, j);
        const int64_t jpos = __shfl_sync(0xffffffffu, pos, j);
        const int jcol = __shfl_sync(0xffffffffu, colbase, j);
        const int jtb = __shfl_sync(0xffffffffu, ep.local, j);
        const uint32_t pinfo = __shfl_sync(0xffffffffu, ep.info, j);
        const T hj = __shfl_sync(0xffffffffu, hspec, j);
        const int jbeg = __shfl_sync(0xffffffffu, beg, j);
        if (t < total1) {
            const ConnEntry<T> en = a.l2_ent[x.l2b + jbeg + k];
            T v;
            if (info_dcode(en.info) != 0) {   // (2,2): V^pn_{c_p c_n, a_p a_n}
                const T w = a.Tpn[jtb + info_tcol(en.info)];
                v = (info_neg(pinfo) ^ info_neg(en.info)) ? -w : w;
            } else {                          // (2,0): neutrons are spectators (n' = n, same 2M)
                v = info_neg(pinfo) ? -hj : hj;
            }
            em.put(a, jpos + k, jcol + en.local, v);
        }
    }
    // 2. p' = p: every same-2M neutron partner of n, L4(n)[0, len)
    const unsigned b2 = __ballot_sync(0xffffffffu, kind == 2 && len > 0);
    if (b2) {
        const int src = __ffs(b2) - 1;
        const int len2 = __shfl_sync(0xffffffffu, len, src);
        const int64_t pos2 = __shfl_sync(0xffffffffu, pos, src);
        const int col2 = __shfl_sync(0xffffffffu, colbase, src);
        const T pval2 = __shfl_sync(0xffffffffu, ep.val, src);
        for (int k = lane; k < len2; k += 32) {
            const ConnEntry<T> en = a.l4_ent[x.l4b + k];
            const int dn = info_dcode(en.info);
            T v;
            if (dn == 2) {                    // (0,4)
                v = en.val;
            } else if (dn == 1) {             // (0,2): protons are spectators
                const T *w = a.Wpn + ((int64_t)info_c(en.info) * S + info_a(en.info)) * S;
                const T h = en.val + sum_over_bits<T>(w, a.p_bits, x.p, a.W);
                v = info_neg(en.info) ? -h : h;
            } else {                          // diagonal
                T h = pval2 + en.val;
                for (int w = 0; w < a.W; ++w) {   // pn diagonal: every occupied proton state with every neutron state
                    uint64_t xp = a.p_bits[(int64_t)x.p * a.W + w];
                    while (xp) {
                        const int kp = 64 * w + __ffsll((long long)xp) - 1;
                        xp &= xp - 1;
                        h += sum_over_bits<T>(a.Dpn + (int64_t)kp * S, a.n_bits, x.n, a.W);
                    }
                }
                v = h;
            }
            em.put(a, pos2 + k, col2 + en.local, v);
        }
    }
    return total;
}

template <class T>
__device__ __forceinline__ void load_partner(const RowArgs<T> &a, const RowCtx &x, int64_t e, bool ok,
                                             ConnEntry<T> &ep, int &kind, int &beg, int &len) {
    if (ok) {
        ep = a.o_ent[e];
        partner_segment<T>(a, x.p, x.n, ep, kind, beg, len);
    } else {
        ep.tgt = 0; ep.local = 0; ep.info = 0; ep.val = 0;
        kind = 0; beg = 0; len = 0;
    }
}

// Fill one row per warp.  One pass over the admissible O2 partners places
// their segments: a partner of 2M slot 0 is preceded by the admissible O4
// partners with a smaller index (its cross rank, capped at their number
// m4), a partner of a higher slot by all m4 of them.  Then the O4 partners
// (one element each) go between, after as many slot-0 O2 elements as their
// own cross rank says.
// Every element (pos, col, value) of a row goes to an emitter: StoreEmit
// writes the CSR arrays; ApplyEmit multiplies by X on the fly (no storage)
// for the expectation values of Fig. 1, observables step.
template <class T>
struct StoreEmit {
    static constexpr int kMinBlocks = 4;   // 64 registers: 32 warps per SM hide the gathers' latency
    __device__ __forceinline__ void init() {}
    __device__ __forceinline__ void put(const RowArgs<T> &a, int64_t pos, int c, T v) {
        a.col[pos] = c;
        a.val[pos] = v;
    }
    __device__ __forceinline__ void end_row(int64_t) {}
    __device__ __forceinline__ void finish(double *) {}
};

// y_i = sum_j O_ij R[j][0..8) accumulated per lane, reduced per row, then
// tot += L[i] * y_i (lane 0); at the end the block's tot goes to part.
template <class T>
struct ApplyEmit {
    static constexpr int kMinBlocks = 2;   // <= 128 registers: two blocks per SM
    const double *R = nullptr;   // right vectors [dim][8], gathered by column
    const double *L = nullptr;   // left vectors [dim][8], one row per row end
    double acc[8], tot[8];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = tot[q] = 0.0;
    }
    __device__ __forceinline__ void put(const RowArgs<T> &, int64_t, int c, T v) {
        const double2 *xc = reinterpret_cast<const double2 *>(R + (int64_t)c * 8);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 t = __ldg(xc + q);
            acc[2 * q] = fma((double)v, t.x, acc[2 * q]);
            acc[2 * q + 1] = fma((double)v, t.y, acc[2 * q + 1]);
        }
    }
    __device__ __forceinline__ void end_row(int64_t r) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            double y = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if ((threadIdx.x & 31) == 0) tot[q] = fma(L[r * 8 + q], y, tot[q]);
            acc[q] = 0.0;
        }
    }
    __device__ __forceinline__ void finish(double *part) {
        __shared__ double red[8][8];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 8; ++q) red[w][q] = tot[q];
        __syncthreads();
        if (threadIdx.x < 8) {
            double t = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i][threadIdx.x];
            part[(int64_t)blockIdx.x * 8 + threadIdx.x] = t;
        }
    }
};

template <class T, class Emit>
__global__ void __launch_bounds__(256, Emit::kMinBlocks) k_rows(const RowArgs<T> *args, const int64_t *row_off, int G, Emit em,
                                              double *part) {
    em.init();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t rows = row_off[G];
    for (int64_t gr = warp; gr < rows; gr += nwarps) {
        const int g = group_of(row_off, G, gr);
        const RowArgs<T> &a = args[g];
        const int64_t r = gr - row_off[g];
        RowCtx x;
        x.p = a.row_p[r];
        x.n = a.row_n[r];
        const int p = x.p, n = x.n;
        x.n_local = a.n_local[n];
        x.l2b = a.l2_ptr[n];
        x.l4b = a.l4_ptr[n];
        const int m4 = o4_count<T>(a, p, n);
        const int64_t row0 = a.row_ptr ? a.row_ptr[r] : 0;   // no output positions when applying
        int64_t out = row0;       // O2 elements placed so far (O4 ones not counted)
        int below = 0;            // O2 elements of the slots below p's own
        int m2 = 0;               // admissible O2 partners of p's own slot
        for_o2<T>(a, p, n, 0, a.nds, [&](int64_t e, bool ok) {
            ConnEntry<T> ep;
            int kind, beg, len;
            load_partner<T>(a, x, e, ok, ep, kind, beg, len);
            const int ds = ok ? info_dslot(ep.info) : -1;
            const int extra = ds > 0 ? m4 : (ds == 0 ? min(a.o_xr[e], m4) : 0);
            unsigned lo_mask = __ballot_sync(0xffffffffu, ok && ds < 0);
            int bl = (lo_mask >> lane) & 1 ? len : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bl += __shfl_xor_sync(0xffffffffu, bl, o);
            below += bl;
            m2 += __popc(__ballot_sync(0xffffffffu, ok && ds == 0));
            out += fill_chunk<T, Emit>(a, x, ep, kind, beg, len, extra, out, em);
        });
        if (m4 > 0) {
            // slot-0 O2 partners: the admissible ones are the first m2 of the
            // slot; the slot starts at entry s0
            const int64_t s0 = a.o_ptr[p] + (a.K == 0 ? 0 : a.oseg2[((int64_t)p * a.nds + a.K - 1) * a.nq + a.nq - 1]);
            const int64_t o4b = a.o4_ptr[p];
            for (int k0 = 0; k0 < m4; k0 += 32) {
                const int k = k0 + lane;
                const bool ok = k < m4;
                ConnEntry<T> e4;
                int lim = 0;          // slot-0 O2 partners before this O4 partner
                if (ok) {
                    e4 = a.o4_ent[o4b + k];
                    lim = min(a.o_xr[o4b + k], m2);
                } else {
                    e4.tgt = 0; e4.local = 0; e4.info = 0; e4.val = 0;
                }
                int lensum = 0;
                for (int i0 = 0; i0 < m2; i0 += 32) {
                    const int i = i0 + lane;
                    int len = 0;
                    if (i < m2) {
                        ConnEntry<T> ep = a.o_ent[s0 + i];
                        int kind, beg;
                        partner_segment<T>(a, p, n, ep, kind, beg, len);
                    }
                    const int incl = warp_incl_scan_i32(len);
                    const int tot = __shfl_sync(0xffffffffu, incl, 31);
                    const int idx = min(max(lim - i0, 0), 32);   // this chunk's partners before k
                    const int part = __shfl_sync(0xffffffffu, incl, idx > 0 ? idx - 1 : 0);
                    lensum += idx >= 32 ? tot : (idx > 0 ? part : 0);
                }
                if (ok) em.put(a, row0 + below + k + lensum, e4.tgt + x.n_local, e4.val);
            }
        }
        em.end_row(r);
    }
    em.finish(part);
}

template <class T>
static RowArgs<T> row_args(Problem *p, const Tables<T> *tab = nullptr, const ConnEntry<T> *ents = nullptr) {
    Connectivity<T> &c = p->conn<T>();
    const Tables<T> &t = tab ? *tab : p->tables<T>();
    SpeciesList &P = p->sp[0], &Nn = p->sp[1];
    RowArgs<T> a{};
    a.dim = p->dim; a.S = p->S; a.W = P.W; a.nq = Nn.nq; a.nds = p->nds; a.K = p->K;
    a.nmax = p->nmax; a.twoM = p->twoM;
    a.row_p = p->d_row_p.ptr; a.row_n = p->d_row_n.ptr; a.p_row_base = p->d_p_row_base.ptr;
    a.p_q = P.d_q.ptr; a.p_twoM = P.d_twoM.ptr; a.n_q = Nn.d_q.ptr; a.n_twoM = Nn.d_twoM.ptr;
    a.n_local = Nn.d_local.ptr; a.p_bits = P.d_bits.ptr; a.n_bits = Nn.d_bits.ptr;
    a.o_ptr = c.outer.ptr; a.o4_ptr = c.outer4.ptr; a.l2_ptr = c.l2.ptr; a.l4_ptr = c.l4.ptr;
    a.o_ent = c.outer.ent; a.o4_ent = c.outer4.ent; a.l2_ent = c.l2.ent; a.l4_ent = c.l4.ent;
    a.o_xr = c.outer.xr;
    if (ents) {  // another operator's entries in the same layout
        a.o_ent = ents; a.o4_ent = ents; a.l2_ent = ents; a.l4_ent = ents;
    }
    a.seg2 = c.seg2.ptr; a.seg4 = c.seg4.ptr; a.qmin2 = c.qmin2.ptr; a.oseg2 = c.oseg2.ptr; a.oseg4 = c.oseg4.ptr;
    a.Upn = t.Upn.ptr; a.Wpn = t.Wpn.ptr; a.Dpn = t.Dpn.ptr; a.Tpn = t.Tpn.ptr;
    return a;
}

static int row_grid(int64_t rows) { return grid_for(rows * 32, 256, sm_count() * 8); }

template <class T>
static void upload_args(const std::vector<RowArgs<T>> &args, const std::vector<int64_t> &row_off,
                        DevBuf<unsigned char> &dargs, DevBuf<int64_t> &doff, cudaStream_t s) {
    dargs.alloc(sizeof(RowArgs<T>) * args.size());
    doff.alloc(row_off.size());
    CI_CUDA(cudaMemcpyAsync(dargs.ptr, args.data(), sizeof(RowArgs<T>) * args.size(), cudaMemcpyHostToDevice, s));
    CI_CUDA(cudaMemcpyAsync(doff.ptr, row_off.data(), sizeof(int64_t) * row_off.size(), cudaMemcpyHostToDevice, s));
}

template <class T>
static void count_group_t(const std::vector<Problem *> &ps, GroupCSR *g, cudaStream_t s) {
    species_filter_group<T>(ps, s);
    g->prec = sizeof(T) == 4 ? 0 : 1;
    g->row_off.assign(1, 0);
    std::vector<RowArgs<T>> args;
    for (Problem *p : ps) {
        g->row_off.push_back(g->row_off.back() + p->dim);
        args.push_back(row_args<T>(p));
    }
    const int64_t rows = g->row_off.back();
    g->row_cnt.alloc(rows);
    for (size_t i = 0; i < ps.size(); ++i) args[i].row_cnt = g->row_cnt.ptr + g->row_off[i];
    if (rows > 0) {
        DevBuf<unsigned char> dargs;
        DevBuf<int64_t> doff;
        upload_args<T>(args, g->row_off, dargs, doff, s);
        launch("k_count_rows", k_count_rows<T>, row_grid(rows), 256, 0, s, (const RowArgs<T> *)dargs.ptr,
               (const int64_t *)doff.ptr, (int)ps.size());
    }
}

void count_group(const std::vector<Problem *> &ps, int prec, GroupCSR *g, cudaStream_t s) {
    if (prec == 0) count_group_t<float>(ps, g, s);
    else count_group_t<double>(ps, g, s);
    // offsets of every row (Eq. 1) and the total per problem
    const int64_t rows = g->row_off.back();
    g->row_ptr.alloc(rows + 1);
    exclusive_scan_i32(g->row_cnt.ptr, rows, g->row_ptr.ptr, ps[0]->scan_scratch, s);
    const std::vector<int64_t> ends = gather_i64(g->row_ptr.ptr, g->row_off, s);
    g->nnz = ends[ps.size()];
    g->nnz_of.resize(ps.size());
    for (size_t i = 0; i < ps.size(); ++i) g->nnz_of[i] = ends[i + 1] - ends[i];
}

template <class T>
static void fill_group_t(const std::vector<Problem *> &ps, GroupCSR *g, cudaStream_t s) {
    std::vector<RowArgs<T>> args;
    for (size_t i = 0; i < ps.size(); ++i) {
        args.push_back(row_args<T>(ps[i]));
        args.back().row_ptr = g->row_ptr.ptr + g->row_off[i];
        args.back().col = g->col.ptr;
        args.back().val = (T *)g->val.ptr;
    }
    const int64_t rows = g->row_off.back();
    if (rows == 0) return;
    DevBuf<unsigned char> dargs;
    DevBuf<int64_t> doff;
    upload_args<T>(args, g->row_off, dargs, doff, s);
    launch("k_fill_rows", k_rows<T, StoreEmit<T>>, row_grid(rows), 256, 0, s, (const RowArgs<T> *)dargs.ptr,
           (const int64_t *)doff.ptr, (int)ps.size(), StoreEmit<T>{}, (double *)nullptr);
}

// Fig. 1, offsets and fill for a counted group: allocate and fill col / val.
void fill_group(const std::vector<Problem *> &ps, GroupCSR *g, cudaStream_t s) {
    g->col.alloc(g->nnz);
    g->val.alloc(g->nnz * (g->prec ? sizeof(double) : sizeof(float)));
    if (g->prec == 0) fill_group_t<float>(ps, g, s);
    else fill_group_t<double>(ps, g, s);
}

// y_i = sum_j H_ij R[j][0..8), each element evaluated on the fly (nothing
// stored), written to Y [dim][8]: the FP64 product of the Ritz refinement.
template <class T>
struct ProductEmit {
    static constexpr int kMinBlocks = 1;
    const double *R = nullptr;   // [dim][8], gathered by column
    double *Y = nullptr;         // [dim][8]
    double acc[8];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    }
    __device__ __forceinline__ void put(const RowArgs<T> &, int64_t, int c, T v) {
        const double2 *xc = reinterpret_cast<const double2 *>(R + (int64_t)c * 8);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 t = __ldg(xc + q);
            acc[2 * q] = fma((double)v, t.x, acc[2 * q]);
            acc[2 * q + 1] = fma((double)v, t.y, acc[2 * q + 1]);
        }
    }
    __device__ __forceinline__ void end_row(int64_t r) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            double y = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
            if ((threadIdx.x & 31) == 0) Y[r * 8 + q] = y;
            acc[q] = 0.0;
        }
    }
    __device__ __forceinline__ void finish(double *) {}
};

void h64_apply(Problem *p, const double *R8, double *Y8, cudaStream_t s) {
    species_filter<double>(p, s);
    if (p->dim == 0) return;
    std::vector<RowArgs<double>> args{row_args<double>(p)};
    std::vector<int64_t> row_off{0, p->dim};
    DevBuf<unsigned char> dargs;
    DevBuf<int64_t> doff;
    upload_args<double>(args, row_off, dargs, doff, s);
    ProductEmit<double> em{};
    em.R = R8;
    em.Y = Y8;
    launch("k_h64_rows", k_rows<double, ProductEmit<double>>, row_grid(p->dim), 256, 0, s,
           (const RowArgs<double> *)dargs.ptr, (const int64_t *)doff.ptr, 1, em, (double *)nullptr);
}

template <class T>
int observable_apply(Problem *p, const Tables<T> &t, const ConnEntry<T> *ents, const double *L8, const double *R8,
                     double *part, cudaStream_t s) {
    std::vector<RowArgs<T>> args{row_args<T>(p, &t, ents)};
    std::vector<int64_t> row_off{0, p->dim};
    if (p->dim == 0) return 0;
    DevBuf<unsigned char> dargs;
    DevBuf<int64_t> doff;
    upload_args<T>(args, row_off, dargs, doff, s);
    ApplyEmit<T> em{};
    em.L = L8;
    em.R = R8;
    const int grid = row_grid(p->dim);
    launch("k_observable_rows", k_rows<T, ApplyEmit<T>>, grid, 256, 0, s, (const RowArgs<T> *)dargs.ptr,
           (const int64_t *)doff.ptr, 1, em, part);
    return grid;
}

template int observable_apply<float>(Problem *, const Tables<float> &, const ConnEntry<float> *, const double *,
                                     const double *, double *, cudaStream_t);
template int observable_apply<double>(Problem *, const Tables<double> &, const ConnEntry<double> *, const double *,
                                      const double *, double *, cudaStream_t);

// BF16 storage with a per-row scale: scale_r = max_j |v_rj| (1 for an
// all-zero row), stored value bf16(v / scale_r) rounded to nearest; one
// warp per row.
__global__ void k_to_bf16_rows(int64_t dim, const int64_t *__restrict__ rp, const float *__restrict__ v32,
                               __nv_bfloat16 *__restrict__ v16, float *__restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < dim; r += nwarps) {
        const int64_t e0 = rp[r], e1 = rp[r + 1];
        float m = 0.f;
        for (int64_t e = e0 + lane; e < e1; e += 32) m = fmaxf(m, fabsf(v32[e]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float sc = m > 0.f ? m : 1.f;
        const float inv = 1.f / sc;
        for (int64_t e = e0 + lane; e < e1; e += 32) v16[e] = __float2bfloat16_rn(v32[e] * inv);
        if (lane == 0) scale[r] = sc;
    }
}

void build_matrix(Problem *p, int vtype, Matrix *m, cudaStream_t s) {
    if (vtype != CI_F32 && vtype != CI_F64 && vtype != CI_BF16_ROWSCALE)
        fail(CI_ERR_INVALID_ARG, "value type %d is not supported by ci_build_H", vtype);
    GroupCSR g;
    count_group({p}, vtype == CI_F64 ? 1 : 0, &g, s);
    fill_group({p}, &g, s);
    m->dim = p->dim;
    m->vtype = vtype;
    m->nnz = g.nnz;
    m->row_ptr = std::move(g.row_ptr);
    m->col = std::move(g.col);
    spmm_prepare(m, s);
    if (vtype != CI_BF16_ROWSCALE) {
        m->val = std::move(g.val);
        return;
    }
    // values filled in FP32, then scaled per row and rounded to bf16
    m->val.alloc((size_t)g.nnz * sizeof(__nv_bfloat16));
    m->row_scale.alloc((size_t)p->dim);
    if (p->dim > 0)
        launch("k_to_bf16_rows", k_to_bf16_rows, row_grid(p->dim), 256, 0, s, p->dim, m->row_ptr.ptr,
               (const float *)g.val.ptr, (__nv_bfloat16 *)m->val.ptr, m->row_scale.ptr);
}

}  // namespace ci
