// Problem set-up: validation, the host planner of the species lists and the
// product basis (Fig. 1, basis step), and the staging of the interaction into
// compact device tables.
#include <algorithm>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>

#include "problem.cuh"

namespace ci {

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

void set_last_error(const std::string &m) { g_last_error = m; }
const char *last_error_cstr() { return g_last_error.c_str(); }

void fail(ci_status s, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    throw Error(s, buf);
}

bool is_device_pointer(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void copy_out(void *dst, const void *src_dev, size_t bytes, cudaStream_t s) {
    if (!dst || bytes == 0) return;
    CI_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDefault, s));
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        CI_CUDA(cudaGetDevice(&dev));
        CI_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    }
    return n;
}

// ------------------------------------------------------------------ TBME source

// Parameters every staging thread needs to fetch V_abcd of one channel.
struct TbmeSrc {
    int S;
    int source;         // CI_TBME_TABLES / CI_TBME_SEED
    int dtype;          // CI_F32 / CI_F64 of the flat table
    const void *flat;   // S^4 entries (tables) or null
    uint64_t seed;
    int channel;        // 0 pp, 1 nn, 2 pn
    const int32_t *twom;
};

__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// g(seed, channel, P, Q) of the counter-based recipe in mfdci.h; the
// integer sum is exact, so the double result is exact.
__device__ double tbme_draw(uint64_t seed, int channel, uint32_t P, uint32_t Q) {
    uint64_t c = ((uint64_t)channel << 32) | ((uint64_t)P << 16) | (uint64_t)Q;
    uint64_t acc = 0;
    for (int k = 0; k < 12; ++k)
        acc += splitmix64_mix(seed + (12ull * c + (uint64_t)(k + 1)) * 0x9E3779B97F4A7C15ull) >> 32;
    return (double)acc * (1.0 / 4294967296.0) - 6.0;
}

// V_abcd of one channel, exact in binary64 (a float table is widened).
__device__ double tbme_fetch(const TbmeSrc &t, int a, int b, int c, int d) {
    if (t.source == CI_TBME_TABLES) {
        int64_t i = (((int64_t)a * t.S + b) * t.S + c) * t.S + d;
        return t.dtype == CI_F32 ? (double)((const float *)t.flat)[i]
                                 : ((const double *)t.flat)[i];
    }
    if (t.twom[a] + t.twom[b] != t.twom[c] + t.twom[d]) return 0.0;
    if (t.channel == 2) {
        uint32_t P = (uint32_t)(a * t.S + b), Q = (uint32_t)(c * t.S + d);
        return P <= Q ? tbme_draw(t.seed, 2, P, Q) : tbme_draw(t.seed, 2, Q, P);
    }
    if (a == b || c == d) return 0.0;
    double s = 1.0;
    if (a > b) { int x = a; a = b; b = x; s = -s; }
    if (c > d) { int x = c; c = d; d = x; s = -s; }
    uint32_t P = (uint32_t)(b * (b - 1) / 2 + a), Q = (uint32_t)(d * (d - 1) / 2 + c);
    return s * (P <= Q ? tbme_draw(t.seed, t.channel, P, Q) : tbme_draw(t.seed, t.channel, Q, P));
}

// Value of V in the table precision: a float table (or draw) rounds to
// nearest float when T = float.
template <class T>
__device__ __forceinline__ T to_prec(double v, const TbmeSrc &t) {
    (void)t;
    return (T)v;
}

// One staging job fills one table of one problem.
//   kind 0, compact blocks: entry e of group g is (row item i, column item j)
//     of the group's lists (items are codes x*S+y); mode 0 (like pairs): row
//     (c,d), column (a,b) -> V_{cd,ab}; mode 1 (pn moves): row (c,a) proton
//     move, column (c',a') neutron move -> V^pn_{c c', a a'}
//   kind 1, spectators: U[(c*S+a)*S+k] = V_{ck,ak}; mode 1: W[(d*S+b)*S+k] = V_{kd,kb}
//   kind 2, pair diagonals: D[a*S+b] = V_abab
//   kind 3, one-body energies: eps[a] (from eps64)
template <class T>
struct StageJob {
    TbmeSrc src;
    int kind, mode, G;
    const int64_t *goff;
    const int32_t *gncol, *grows, *gcols, *items;
    const double *eps64;
    int64_t total;
    T *out;
};

template <class T>
__device__ void stage_one(const StageJob<T> &j, int64_t e) {
    const TbmeSrc &t = j.src;
    if (j.kind == 0) {
        int lo = 0, hi = j.G - 1;
        while (lo < hi) {  // last group with goff <= e
            int mid = (lo + hi + 1) >> 1;
            if (j.goff[mid] <= e) lo = mid; else hi = mid - 1;
        }
        int64_t r = e - j.goff[lo];
        int n = j.gncol[lo];
        int i = (int)(r / n), k = (int)(r % n);
        int pr = j.items[j.grows[lo] + i], pc = j.items[j.gcols[lo] + k];
        int x1 = pr / t.S, y1 = pr % t.S, x2 = pc / t.S, y2 = pc % t.S;
        double v = j.mode == 0 ? tbme_fetch(t, x1, y1, x2, y2) : tbme_fetch(t, x1, x2, y1, y2);
        j.out[e] = to_prec<T>(v, t);
    } else if (j.kind == 1) {
        int k = (int)(e % t.S);
        int a = (int)((e / t.S) % t.S);
        int c = (int)(e / ((int64_t)t.S * t.S));
        double v = j.mode ? tbme_fetch(t, k, c, k, a) : tbme_fetch(t, c, k, a, k);
        j.out[e] = to_prec<T>(v, t);
    } else if (j.kind == 2) {
        int a = (int)(e / t.S), b = (int)(e % t.S);
        j.out[e] = to_prec<T>(tbme_fetch(t, a, b, a, b), t);
    } else {
        j.out[e] = (T)j.eps64[e];
    }
}

template <class T>
__global__ void k_stage(const StageJob<T> *jobs, const int64_t *job_off, int njobs) {
    const int64_t total = job_off[njobs];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (job_off[mid] <= e) lo = mid; else hi = mid - 1;
        }
        stage_one<T>(jobs[lo], e - job_off[lo]);
    }
}

// ------------------------------------------------------------------ pair maps

// Groups of a compact table: group g has rows items[grp_rows[g] ..] and
// columns items[grp_cols[g] ..], stored row-major from grp_off[g].
struct PairGroups {
    std::vector<int64_t> grp_off;   // [G+1] compact offsets
    std::vector<int32_t> grp_ncol;  // [G]
    std::vector<int32_t> grp_rows;  // [G] start of the row items
    std::vector<int32_t> grp_cols;  // [G] start of the column items
    std::vector<int32_t> items;     // codes x*S+y
    std::vector<int32_t> row, col;  // [S*S]: row offset / column index, -1 if none
};

// like pairs a<b grouped by m_a + m_b (rows = columns = the group's pairs)
static PairGroups make_like_pairs(const std::vector<int32_t> &twom) {
    int S = (int)twom.size();
    std::map<int, std::vector<int32_t>> by_m;
    for (int a = 0; a < S; ++a)
        for (int b = a + 1; b < S; ++b) by_m[twom[a] + twom[b]].push_back(a * S + b);
    PairGroups g;
    g.row.assign((size_t)S * S, -1);
    g.col.assign((size_t)S * S, -1);
    int64_t off = 0;
    for (auto &kv : by_m) {
        auto &v = kv.second;
        g.grp_off.push_back(off);
        g.grp_ncol.push_back((int32_t)v.size());
        g.grp_rows.push_back((int32_t)g.items.size());
        g.grp_cols.push_back((int32_t)g.items.size());
        for (size_t i = 0; i < v.size(); ++i) {
            g.row[v[i]] = (int32_t)(off + (int64_t)i * (int64_t)v.size());
            g.col[v[i]] = (int32_t)i;
            g.items.push_back(v[i]);
        }
        off += (int64_t)v.size() * (int64_t)v.size();
    }
    g.grp_off.push_back(off);
    return g;
}

// one-particle moves a -> c (c != a) grouped by D = 2m_c - 2m_a; the block
// of D has the proton moves of D as rows and the neutron moves of -D as
// columns (total M is conserved).  row[c*S+a] = offset of the move's row,
// col[c*S+a] = index of the move in its own group (its column index).
static PairGroups make_transitions(const std::vector<int32_t> &twom) {
    int S = (int)twom.size();
    std::map<int, std::vector<int32_t>> by_d;
    for (int c = 0; c < S; ++c)
        for (int a = 0; a < S; ++a)
            if (c != a) by_d[twom[c] - twom[a]].push_back(c * S + a);
    PairGroups g;
    g.row.assign((size_t)S * S, -1);
    g.col.assign((size_t)S * S, -1);
    std::map<int, int32_t> start;
    for (auto &kv : by_d) {
        start[kv.first] = (int32_t)g.items.size();
        for (size_t i = 0; i < kv.second.size(); ++i) {
            g.col[kv.second[i]] = (int32_t)i;
            g.items.push_back(kv.second[i]);
        }
    }
    int64_t off = 0;
    for (auto &kv : by_d) {
        auto it = by_d.find(-kv.first);
        if (it == by_d.end()) continue;
        int32_t nr = (int32_t)kv.second.size(), nc = (int32_t)it->second.size();
        g.grp_off.push_back(off);
        g.grp_ncol.push_back(nc);
        g.grp_rows.push_back(start[kv.first]);
        g.grp_cols.push_back(start[-kv.first]);
        for (int32_t i = 0; i < nr; ++i) g.row[kv.second[i]] = (int32_t)(off + (int64_t)i * nc);
        off += (int64_t)nr * nc;
    }
    g.grp_off.push_back(off);
    return g;
}

// ------------------------------------------------------------------ create

void problem_create(const ci_problem_desc *d, Problem *p) {
    if (!d) fail(CI_ERR_INVALID_ARG, "desc is NULL");
    if (d->n_sp < 1 || d->n_sp > 64 * kMaxWords)
        fail(CI_ERR_INVALID_ARG, "n_sp must be 1..%d (got %d)", 64 * kMaxWords, d->n_sp);
    if (!d->sp_N || !d->sp_twom || !d->sp_energy)
        fail(CI_ERR_INVALID_ARG, "sp_N, sp_twom and sp_energy are required");
    if (d->Z < 0 || d->N < 0 || d->Z > kMaxA || d->N > kMaxA || d->Z > d->n_sp || d->N > d->n_sp)
        fail(CI_ERR_INVALID_ARG, "Z and N must be 0..min(S,%d)", kMaxA);
    if (d->nmax < -1) fail(CI_ERR_INVALID_ARG, "nmax must be >= -1");
    if (d->nmax > 31) fail(CI_ERR_CAPACITY, "nmax above 31 is not supported");
    if (d->tbme_source != CI_TBME_TABLES && d->tbme_source != CI_TBME_SEED)
        fail(CI_ERR_INVALID_ARG, "tbme_source must be CI_TBME_TABLES or CI_TBME_SEED");
    if (d->tbme_source == CI_TBME_TABLES) {
        if (!d->v_pp || !d->v_nn || !d->v_pn) fail(CI_ERR_INVALID_ARG, "v_pp, v_nn, v_pn are required");
        if (d->tbme_dtype != CI_F32 && d->tbme_dtype != CI_F64)
            fail(CI_ERR_INVALID_ARG, "tbme_dtype must be CI_F32 or CI_F64");
    }
    p->S = d->n_sp;
    p->sp_N.assign(d->sp_N, d->sp_N + d->n_sp);
    p->sp_twom.assign(d->sp_twom, d->sp_twom + d->n_sp);
    p->sp_energy.assign(d->sp_energy, d->sp_energy + d->n_sp);
    for (int a = 0; a < p->S; ++a) {
        if (p->sp_N[a] < 0) fail(CI_ERR_INVALID_ARG, "sp_N[%d] < 0", a);
        if ((p->sp_twom[a] & 1) == 0) fail(CI_ERR_INVALID_ARG, "sp_twom[%d] must be odd", a);
        p->K = std::max(p->K, std::abs(p->sp_twom[a]));
    }
    if (p->K > 63) fail(CI_ERR_CAPACITY, "|2m| above 63 is not supported");
    p->nds = 2 * p->K + 1;
    p->Z = d->Z; p->N = d->N; p->nmax = d->nmax; p->twoM = d->twoM;
    p->tbme_source = d->tbme_source;
    p->tbme_seed = d->tbme_seed;
    p->tbme_dtype = d->tbme_dtype;

    cudaStream_t s = current_stream();
    if (p->tbme_source == CI_TBME_TABLES) {
        size_t esz = p->tbme_dtype == CI_F32 ? 4 : 8;
        size_t bytes = esz * (size_t)p->S * p->S * p->S * p->S;
        const void *src[3] = {d->v_pp, d->v_nn, d->v_pn};
        for (int c = 0; c < 3; ++c) {
            p->flat[c].alloc(bytes);
            CI_CUDA(cudaMemcpyAsync(p->flat[c].ptr, src[c], bytes, cudaMemcpyDefault, s));
        }
    }
    PairGroups lg = make_like_pairs(p->sp_twom), tg = make_transitions(p->sp_twom);
    for (int32_t c : tg.col)
        if (c >= kMaxTcol) fail(CI_ERR_CAPACITY, "a 2m-transfer class holds more than %d one-particle moves", kMaxTcol);
    p->like_row.upload(lg.row, s); p->like_col.upload(lg.col, s);
    p->tr_base.upload(tg.row, s); p->tr_idx.upload(tg.col, s);
    p->like_size = lg.grp_off.back();
    p->tr_size = tg.grp_off.back();
    p->like_G = (int)lg.grp_ncol.size();
    p->tr_G = (int)tg.grp_ncol.size();
    p->lg_off.upload(lg.grp_off, s); p->lg_ncol.upload(lg.grp_ncol, s); p->lg_rows.upload(lg.grp_rows, s);
    p->lg_cols.upload(lg.grp_cols, s); p->lg_items.upload(lg.items, s);
    p->tg_off.upload(tg.grp_off, s); p->tg_ncol.upload(tg.grp_ncol, s); p->tg_rows.upload(tg.grp_rows, s);
    p->tg_cols.upload(tg.grp_cols, s); p->tg_items.upload(tg.items, s);
    p->d_twom.upload(p->sp_twom, s);
    p->d_eps.upload(p->sp_energy, s);
    CI_CUDA(cudaStreamSynchronize(s));
}

// Stage the tables of precision T of every problem in ps that lacks them,
// in one launch.
// Staging jobs that fill the tables t of problem p from the TBME sources
// src[pp, nn, pn] and the one-body energies eps64 (device, S doubles).
template <class T>
static void add_stage_jobs(Problem *p, Tables<T> &t, const TbmeSrc src[3], const double *eps64,
                           std::vector<StageJob<T>> &jobs, std::vector<int64_t> &off) {
    auto add = [&](const StageJob<T> &j) {
        if (j.total <= 0) return;
        jobs.push_back(j);
        off.push_back(off.back() + j.total);
    };
    const int S = p->S;
    const int64_t S3 = (int64_t)S * S * S, S2 = (int64_t)S * S;
    t.eps.alloc(S);
    t.Cpp.alloc(p->like_size); t.Cnn.alloc(p->like_size); t.Tpn.alloc(p->tr_size);
    t.Upp.alloc(S3); t.Unn.alloc(S3); t.Upn.alloc(S3); t.Wpn.alloc(S3);
    t.Dpp.alloc(S2); t.Dnn.alloc(S2); t.Dpn.alloc(S2);
    StageJob<T> j{};
    j.kind = 0; j.mode = 0; j.G = p->like_G; j.goff = p->lg_off.ptr; j.gncol = p->lg_ncol.ptr;
    j.grows = p->lg_rows.ptr; j.gcols = p->lg_cols.ptr; j.items = p->lg_items.ptr; j.total = p->like_size;
    j.src = src[0]; j.out = t.Cpp.ptr; add(j);
    j.src = src[1]; j.out = t.Cnn.ptr; add(j);
    j.mode = 1; j.G = p->tr_G; j.goff = p->tg_off.ptr; j.gncol = p->tg_ncol.ptr; j.grows = p->tg_rows.ptr;
    j.gcols = p->tg_cols.ptr; j.items = p->tg_items.ptr; j.total = p->tr_size; j.src = src[2]; j.out = t.Tpn.ptr;
    add(j);
    StageJob<T> k{};
    k.kind = 1; k.total = S3;
    k.src = src[0]; k.mode = 0; k.out = t.Upp.ptr; add(k);
    k.src = src[1]; k.out = t.Unn.ptr; add(k);
    k.src = src[2]; k.out = t.Upn.ptr; add(k);
    k.mode = 1; k.out = t.Wpn.ptr; add(k);
    StageJob<T> d{};
    d.kind = 2; d.total = S2;
    d.src = src[0]; d.out = t.Dpp.ptr; add(d);
    d.src = src[1]; d.out = t.Dnn.ptr; add(d);
    d.src = src[2]; d.out = t.Dpn.ptr; add(d);
    StageJob<T> e{};
    e.kind = 3; e.total = S; e.src = src[0]; e.eps64 = eps64; e.out = t.eps.ptr; add(e);
}

template <class T>
static void run_stage_jobs(const std::vector<StageJob<T>> &jobs, const std::vector<int64_t> &off, cudaStream_t s) {
    if (jobs.empty()) return;
    DevBuf<StageJob<T>> djobs((size_t)jobs.size());
    DevBuf<int64_t> doff(off.size());
    CI_CUDA(cudaMemcpyAsync(djobs.ptr, jobs.data(), sizeof(StageJob<T>) * jobs.size(), cudaMemcpyHostToDevice, s));
    CI_CUDA(cudaMemcpyAsync(doff.ptr, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, s));
    launch("k_stage", k_stage<T>, grid_for(off.back(), 256, sm_count() * 16), 256, 0, s, (const StageJob<T> *)djobs.ptr,
           (const int64_t *)doff.ptr, (int)jobs.size());
}

template <class T>
void stage_tables_group(const std::vector<Problem *> &ps, cudaStream_t s) {
    std::vector<StageJob<T>> jobs;
    std::vector<int64_t> off(1, 0);
    std::vector<Problem *> todo;
    for (Problem *p : ps) {
        Tables<T> &t = p->tables<T>();
        if (t.ready) continue;
        todo.push_back(p);
        TbmeSrc src[3];
        for (int c = 0; c < 3; ++c) {
            src[c].S = p->S;
            src[c].source = p->tbme_source;
            src[c].dtype = p->tbme_dtype;
            src[c].flat = p->flat[c].ptr;
            src[c].seed = p->tbme_seed;
            src[c].channel = c;
            src[c].twom = p->d_twom.ptr;
        }
        add_stage_jobs<T>(p, t, src, p->d_eps.ptr, jobs, off);
    }
    run_stage_jobs<T>(jobs, off, s);
    for (Problem *p : todo) p->tables<T>().ready = true;
}

// Tables of a two-body operator with the seeded TBMEs of `seed` (the
// recipe of CI_TBME_SEED) and no one-body part.
template <class T>
void stage_operator_tables(Problem *p, uint64_t seed, Tables<T> &t, const double *zero_eps, cudaStream_t s) {
    std::vector<StageJob<T>> jobs;
    std::vector<int64_t> off(1, 0);
    TbmeSrc src[3];
    for (int c = 0; c < 3; ++c) {
        src[c].S = p->S;
        src[c].source = CI_TBME_SEED;
        src[c].dtype = CI_F64;
        src[c].flat = nullptr;
        src[c].seed = seed;
        src[c].channel = c;
        src[c].twom = p->d_twom.ptr;
    }
    add_stage_jobs<T>(p, t, src, zero_eps, jobs, off);
    run_stage_jobs<T>(jobs, off, s);
    t.ready = true;
}

template void stage_operator_tables<float>(Problem *, uint64_t, Tables<float> &, const double *, cudaStream_t);
template void stage_operator_tables<double>(Problem *, uint64_t, Tables<double> &, const double *, cudaStream_t);
template void stage_tables_group<float>(const std::vector<Problem *> &, cudaStream_t);
template void stage_tables_group<double>(const std::vector<Problem *> &, cudaStream_t);

// ------------------------------------------------------------------ species lists

// Enumerate every A-subset of the s.p. states with excess quanta <= nmax
// (Sec. 2.1: a determinant is a bit string with A ones), pruning branches
// whose lightest completion already exceeds the cut.
static void enumerate_species(const Problem *p, int A, SpeciesList *L) {
    const int S = p->S;
    L->A = A;
    L->W = (S + 63) / 64;
    // suffix_min[o][r]: smallest sum of r shells among states o..S-1
    std::vector<std::vector<int>> suffix_min(S + 1, std::vector<int>(A + 1, 1 << 28));
    for (int o = S; o >= 0; --o) {
        std::vector<int> v(p->sp_N.begin() + o, p->sp_N.end());
        std::sort(v.begin(), v.end());
        int acc = 0;
        suffix_min[o][0] = 0;
        for (int r = 1; r <= A && r <= (int)v.size(); ++r) { acc += v[r - 1]; suffix_min[o][r] = acc; }
    }
    const int nmin = suffix_min[0][A];
    const int64_t cap = 1ll << 26;
    struct Tmp { int twoM, q; uint64_t w[kMaxWords]; uint8_t occ[kMaxA]; };
    struct Walk {
        const Problem *p;
        const std::vector<std::vector<int>> &suffix_min;
        int S, A, nmin;
        int64_t cap;
        std::vector<Tmp> out;
        uint8_t occ[kMaxA];
        void rec(int start, int depth, int Nsum, int msum) {
            if (depth == A) {
                Tmp t;
                t.twoM = msum;
                t.q = Nsum - nmin;
                for (int w = 0; w < kMaxWords; ++w) t.w[w] = 0;
                for (int k = 0; k < A; ++k) { t.occ[k] = occ[k]; t.w[occ[k] >> 6] |= 1ull << (occ[k] & 63); }
                out.push_back(t);
                if ((int64_t)out.size() > cap) fail(CI_ERR_CAPACITY, "species list larger than 2^26 determinants");
                return;
            }
            for (int o = start; o <= S - (A - depth); ++o) {
                if (p->nmax >= 0) {
                    int lb = Nsum + p->sp_N[o] + suffix_min[o + 1][A - depth - 1];
                    if (lb - nmin > p->nmax) continue;
                }
                occ[depth] = (uint8_t)o;
                rec(o + 1, depth + 1, Nsum + p->sp_N[o], msum + p->sp_twom[o]);
            }
        }
    } walk{p, suffix_min, S, A, nmin, cap, {}, {}};
    walk.rec(0, 0, 0, 0);
    std::vector<Tmp> &out = walk.out;
    std::sort(out.begin(), out.end(), [](const Tmp &x, const Tmp &y) {
        if (x.twoM != y.twoM) return x.twoM < y.twoM;
        if (x.q != y.q) return x.q < y.q;
        for (int w = kMaxWords - 1; w > 0; --w)
            if (x.w[w] != y.w[w]) return x.w[w] < y.w[w];
        return x.w[0] < y.w[0];
    });
    L->n = (int64_t)out.size();
    L->bits.assign((size_t)L->n * L->W, 0);
    L->q.resize(L->n); L->twoM.resize(L->n); L->local.resize(L->n);
    L->occ.assign((size_t)L->n * (A ? A : 1), 0);
    for (int64_t i = 0; i < L->n; ++i) {
        for (int w = 0; w < L->W; ++w) L->bits[i * L->W + w] = out[i].w[w];
        L->q[i] = out[i].q;
        L->twoM[i] = out[i].twoM;
        for (int k = 0; k < A; ++k) L->occ[i * A + k] = out[i].occ[k];
    }
    // 2M blocks and q prefixes
    L->nq = p->nmax >= 0 ? p->nmax + 1 : 1;
    if (L->n == 0) { L->nblk = 0; L->blk_start.assign(1, 0); return; }
    L->m2min = L->twoM.front();
    L->nblk = (L->twoM.back() - L->m2min) / 2 + 1;
    L->blk_start.assign(L->nblk + 1, 0);
    L->blk_qend.assign((size_t)L->nblk * L->nq, 0);
    for (int64_t i = 0; i < L->n; ++i) L->blk_start[(L->twoM[i] - L->m2min) / 2 + 1]++;
    for (int b = 0; b < L->nblk; ++b) L->blk_start[b + 1] += L->blk_start[b];
    for (int b = 0; b < L->nblk; ++b) {
        int64_t i = L->blk_start[b];
        for (int c = 0; c < L->nq; ++c) {
            if (p->nmax >= 0) { while (i < L->blk_start[b + 1] && L->q[i] <= c) ++i; }
            else i = L->blk_start[b + 1];
            L->blk_qend[(size_t)b * L->nq + c] = i;
        }
        for (int64_t j = L->blk_start[b]; j < L->blk_start[b + 1]; ++j)
            L->local[j] = (int32_t)(j - L->blk_start[b]);
    }
}

// row -> (p, n): p by binary search over p_row_base, n from p's block
__global__ void k_row_map(int64_t dim, int64_t nP, const int64_t *p_row_base,
                          const int64_t *p_nstart, int32_t *row_p, int32_t *row_n) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < dim;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nP - 1;
        while (lo < hi) {  // last p with p_row_base[p] <= r
            int64_t mid = (lo + hi + 1) >> 1;
            if (p_row_base[mid] <= r) lo = mid; else hi = mid - 1;
        }
        row_p[r] = (int32_t)lo;
        row_n[r] = (int32_t)(p_nstart[lo] + (r - p_row_base[lo]));
    }
}

void enumerate_basis(Problem *p, cudaStream_t s) {
    if (p->enumerated) return;
    enumerate_species(p, p->Z, &p->sp[0]);
    if (p->N == p->Z) {  // both species draw from the same s.p. table
        SpeciesList &a = p->sp[0], &b = p->sp[1];
        b.A = a.A; b.W = a.W; b.n = a.n; b.bits = a.bits; b.q = a.q; b.twoM = a.twoM; b.occ = a.occ;
        b.local = a.local; b.m2min = a.m2min; b.nblk = a.nblk; b.nq = a.nq; b.blk_start = a.blk_start;
        b.blk_qend = a.blk_qend;
    } else {
        enumerate_species(p, p->N, &p->sp[1]);
    }
    SpeciesList &P = p->sp[0], &Nn = p->sp[1];
    p->p_row_base.assign(P.n + 1, 0);
    std::vector<int64_t> &p_nstart = p->p_nstart;
    p_nstart.assign(P.n ? P.n : 1, 0);
    for (int64_t i = 0; i < P.n; ++i) {
        int b = Nn.block_of(p->twoM - P.twoM[i]);
        int64_t cnt = 0;
        if (b >= 0) {
            p_nstart[i] = Nn.blk_start[b];
            if (p->nmax >= 0) {
                int c = p->nmax - P.q[i];
                if (c >= 0) cnt = Nn.blk_qend[(size_t)b * Nn.nq + std::min(c, Nn.nq - 1)] - Nn.blk_start[b];
            } else {
                cnt = Nn.blk_start[b + 1] - Nn.blk_start[b];
            }
        }
        p->p_row_base[i + 1] = p->p_row_base[i] + cnt;
    }
    p->dim = P.n ? p->p_row_base[P.n] : 0;
    if (p->dim > (int64_t)INT32_MAX) fail(CI_ERR_CAPACITY, "basis dimension above 2^31-1");
    for (int sp = 0; sp < 2; ++sp) {
        SpeciesList &L = p->sp[sp];
        L.d_bits.upload(L.bits, s);
        L.d_q.upload(L.q, s);
        L.d_twoM.upload(L.twoM, s);
        L.d_local.upload(L.local, s);
        L.d_occ.upload(L.occ, s);
        L.d_blk_start.upload(L.blk_start, s);
    }
    p->d_p_row_base.upload(p->p_row_base, s);
    p->d_p_nstart.upload(p_nstart, s);
    p->d_row_p.alloc(p->dim);
    p->d_row_n.alloc(p->dim);
    if (p->dim > 0) {
        launch("k_row_map", k_row_map, grid_for(p->dim, 256), 256, 0, s, p->dim, P.n, p->d_p_row_base.ptr, p->d_p_nstart.ptr,
                                                         p->d_row_p.ptr, p->d_row_n.ptr);
        CI_CHECK_LAUNCH();
    }
    p->enumerated = true;
}

}  // namespace ci
