// extern "C" entry points of mfdci.h: argument checks, handle ownership and
// status conversion around the internal steps.
#include <cstring>
#include <memory>
#include <mutex>

#include "problem.cuh"

namespace ci {
const char *last_error_cstr();
}

using namespace ci;

static cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

template <class T>
static void export_conn(const Problem &P, int species, int64_t *ptr, int32_t *idx, int8_t *d, int64_t cap,
                        int64_t *total) {
    const Connectivity<T> &c = const_cast<Problem &>(P).conn<T>();
    // species 0: the proton list; species 1: the union of the neutron lists
    // L2 and L4 (the neutron pairs kept), merged per row in ascending order.
    if (species == 0) {
        // O2 (d <= 2) and O4 (d = 4, same 2M) merged per row by partner index
        const ConnList<T> &A = c.outer, &B = c.outer4;
        const int64_t n = P.sp[0].n;
        std::vector<int64_t> pa(n + 1), pb(n + 1);
        CI_CUDA(cudaMemcpy(pa.data(), A.ptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        CI_CUDA(cudaMemcpy(pb.data(), B.ptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        for (auto &x : pa) x -= A.first;
        for (auto &x : pb) x -= B.first;
        const int64_t tot = A.total + B.total;
        if (total) *total = tot;
        if (ptr)
            for (int64_t i = 0; i <= n; ++i) ptr[i] = pa[i] + pb[i];
        if (!idx && !d) return;
        if (cap < tot) fail(CI_ERR_CAPACITY, "cap below the entry count");
        std::vector<ConnEntry<T>> ea(A.total), eb(B.total);
        std::vector<int32_t> ta(A.total), tb(B.total);
        if (A.total) {
            CI_CUDA(cudaMemcpy(ea.data(), A.ent + A.first, A.total * sizeof(ConnEntry<T>), cudaMemcpyDeviceToHost));
            CI_CUDA(cudaMemcpy(ta.data(), A.tgt + A.first, A.total * sizeof(int32_t), cudaMemcpyDeviceToHost));
        }
        if (B.total) {
            CI_CUDA(cudaMemcpy(eb.data(), B.ent + B.first, B.total * sizeof(ConnEntry<T>), cudaMemcpyDeviceToHost));
            CI_CUDA(cudaMemcpy(tb.data(), B.tgt + B.first, B.total * sizeof(int32_t), cudaMemcpyDeviceToHost));
        }
        int64_t o = 0;
        for (int64_t s = 0; s < n; ++s) {
            int64_t i = pa[s], j = pb[s];
            while (i < pa[s + 1] || j < pb[s + 1]) {
                const bool takeA = j >= pb[s + 1] || (i < pa[s + 1] && ta[i] < tb[j]);
                const int32_t t = takeA ? ta[i] : tb[j];
                const int dc = info_dcode(takeA ? ea[i].info : eb[j].info);
                if (idx) idx[o] = t;
                if (d) d[o] = (int8_t)(2 * dc);
                ++o;
                if (takeA) ++i; else ++j;
            }
        }
        return;
    }
    int64_t n = P.sp[1].n;
    std::vector<int64_t> p2(n + 1), p4(n + 1);
    CI_CUDA(cudaMemcpy(p2.data(), c.l2.ptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    CI_CUDA(cudaMemcpy(p4.data(), c.l4.ptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    for (auto &x : p2) x -= c.l2.first;
    for (auto &x : p4) x -= c.l4.first;
    std::vector<ConnEntry<T>> e2(c.l2.total), e4(c.l4.total);
    if (c.l2.total)
        CI_CUDA(cudaMemcpy(e2.data(), c.l2.ent + c.l2.first, c.l2.total * sizeof(ConnEntry<T>), cudaMemcpyDeviceToHost));
    if (c.l4.total)
        CI_CUDA(cudaMemcpy(e4.data(), c.l4.ent + c.l4.first, c.l4.total * sizeof(ConnEntry<T>), cudaMemcpyDeviceToHost));
    std::vector<int64_t> hp(n + 1, 0);
    std::vector<int32_t> hi;
    std::vector<int8_t> hd;
    for (int64_t s = 0; s < n; ++s) {
        // L4 holds the same-2M partners with d <= 4, L2 all d <= 2: merge,
        // dropping L2's same-2M entries (also in L4)
        int64_t i = p2[s], j = p4[s];
        while (i < p2[s + 1] || j < p4[s + 1]) {
            bool take4;
            if (i >= p2[s + 1]) take4 = true;
            else if (j >= p4[s + 1]) take4 = false;
            else take4 = e4[j].tgt <= e2[i].tgt;
            if (take4) {
                if (i < p2[s + 1] && e2[i].tgt == e4[j].tgt) ++i;
                hi.push_back(e4[j].tgt); hd.push_back((int8_t)(2 * info_dcode(e4[j].info))); ++j;
            } else {
                hi.push_back(e2[i].tgt); hd.push_back((int8_t)(2 * info_dcode(e2[i].info))); ++i;
            }
        }
        hp[s + 1] = (int64_t)hi.size();
    }
    if (total) *total = (int64_t)hi.size();
    if (ptr) std::memcpy(ptr, hp.data(), hp.size() * sizeof(int64_t));
    if (!idx && !d) return;
    if (cap < (int64_t)hi.size()) fail(CI_ERR_CAPACITY, "cap below the entry count");
    if (idx) std::memcpy(idx, hi.data(), hi.size() * sizeof(int32_t));
    if (d) std::memcpy(d, hd.data(), hd.size());
}

extern "C" {

const char *ci_last_error(void) { return last_error_cstr(); }

const char *ci_status_string(ci_status s) {
    switch (s) {
        case CI_OK: return "CI_OK";
        case CI_ERR_INVALID_ARG: return "CI_ERR_INVALID_ARG";
        case CI_ERR_OOM: return "CI_ERR_OOM";
        case CI_ERR_CUDA: return "CI_ERR_CUDA";
        case CI_ERR_CAPACITY: return "CI_ERR_CAPACITY";
        case CI_ERR_TIMEOUT: return "CI_ERR_TIMEOUT";
        case CI_NOT_READY: return "CI_NOT_READY";
        case CI_ERR_CANCELLED: return "CI_ERR_CANCELLED";
        case CI_ERR_INTERNAL: return "CI_ERR_INTERNAL";
        case CI_ERR_NOT_CONVERGED: return "CI_ERR_NOT_CONVERGED";
        case CI_ERR_STATE: return "CI_ERR_STATE";
    }
    return "CI_UNKNOWN";
}

const char *ci_version(void) { return "mfdci 0.1 (sm_103a)"; }

ci_status ci_problem_create(const ci_problem_desc *desc, ci_problem **out) {
    return guard([&] {
        if (!out) fail(CI_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        std::unique_ptr<ci_problem> p(new ci_problem());
        problem_create(desc, &p->impl);
        *out = p.release();
    });
}

void ci_problem_destroy(ci_problem *p) {
    if (!p) return;
    HandleRelease hr;
    delete p;
}

ci_status ci_enumerate_basis(ci_problem *p, int64_t *dim, void *stream) {
    return guard([&] {
        StreamScope scope(as_stream(stream));
        if (!p) fail(CI_ERR_INVALID_ARG, "problem is NULL");
        enumerate_basis(&p->impl, as_stream(stream));
        if (dim) *dim = p->impl.dim;
    });
}

ci_status ci_species_size(const ci_problem *p, int32_t species, int64_t *n, int32_t *words) {
    return guard([&] {
        if (!p || species < 0 || species > 1) fail(CI_ERR_INVALID_ARG, "bad problem or species");
        if (!p->impl.enumerated) fail(CI_ERR_STATE, "call ci_enumerate_basis first");
        if (n) *n = p->impl.sp[species].n;
        if (words) *words = p->impl.sp[species].W;
    });
}

ci_status ci_get_species(const ci_problem *p, int32_t species, uint64_t *bits, int32_t *q, int32_t *twoM,
                         int64_t cap) {
    return guard([&] {
        if (!p || species < 0 || species > 1) fail(CI_ERR_INVALID_ARG, "bad problem or species");
        if (!p->impl.enumerated) fail(CI_ERR_STATE, "call ci_enumerate_basis first");
        const SpeciesList &L = p->impl.sp[species];
        if (cap < L.n) fail(CI_ERR_CAPACITY, "cap %lld < %lld", (long long)cap, (long long)L.n);
        if (bits) std::memcpy(bits, L.bits.data(), L.bits.size() * sizeof(uint64_t));
        if (q) std::memcpy(q, L.q.data(), L.q.size() * sizeof(int32_t));
        if (twoM) std::memcpy(twoM, L.twoM.data(), L.twoM.size() * sizeof(int32_t));
    });
}

ci_status ci_get_basis(const ci_problem *p, int32_t *p_idx, int32_t *n_idx, int64_t cap) {
    return guard([&] {
        if (!p) fail(CI_ERR_INVALID_ARG, "problem is NULL");
        const Problem &P = p->impl;
        if (!P.enumerated) fail(CI_ERR_STATE, "call ci_enumerate_basis first");
        if (cap < P.dim) fail(CI_ERR_CAPACITY, "cap %lld < dim %lld", (long long)cap, (long long)P.dim);
        if (p_idx) CI_CUDA(cudaMemcpy(p_idx, P.d_row_p.ptr, P.dim * sizeof(int32_t), cudaMemcpyDefault));
        if (n_idx) CI_CUDA(cudaMemcpy(n_idx, P.d_row_n.ptr, P.dim * sizeof(int32_t), cudaMemcpyDefault));
    });
}

ci_status ci_species_filter(ci_problem *p, void *stream) {
    return guard([&] {
        StreamScope scope(as_stream(stream));
        if (!p) fail(CI_ERR_INVALID_ARG, "problem is NULL");
        enumerate_basis(&p->impl, as_stream(stream));
        species_filter<float>(&p->impl, as_stream(stream));
    });
}

ci_status ci_get_species_conn(const ci_problem *p, int32_t species, int64_t *ptr, int32_t *idx, int8_t *d,
                              int64_t cap, int64_t *total) {
    return guard([&] {
        if (!p || species < 0 || species > 1) fail(CI_ERR_INVALID_ARG, "bad problem or species");
        const Problem &P = p->impl;
        if (P.c32.ready) export_conn<float>(P, species, ptr, idx, d, cap, total);
        else if (P.c64.ready) export_conn<double>(P, species, ptr, idx, d, cap, total);
        else fail(CI_ERR_STATE, "call ci_species_filter first");
    });
}

ci_status ci_count_nnz(ci_problem *p, int64_t *nnz, int32_t *row_cnt, void *stream) {
    return guard([&] {
        StreamScope scope(as_stream(stream));
        if (!p) fail(CI_ERR_INVALID_ARG, "problem is NULL");
        cudaStream_t s = as_stream(stream);
        Problem &P = p->impl;
        enumerate_basis(&P, s);
        GroupCSR g;
        count_group({&P}, P.c64.ready && !P.c32.ready ? 1 : 0, &g, s);
        if (row_cnt) copy_out(row_cnt, g.row_cnt.ptr, P.dim * sizeof(int32_t), s);
        CI_CUDA(cudaStreamSynchronize(s));
        if (nnz) *nnz = g.nnz;
    });
}

ci_status ci_exclusive_scan(const int32_t *counts, int64_t n, int64_t *offsets, void *stream) {
    return guard([&] {
        StreamScope scope(as_stream(stream));
        if (n < 0) fail(CI_ERR_INVALID_ARG, "n < 0");
        if (!offsets || (n > 0 && !counts)) fail(CI_ERR_INVALID_ARG, "counts/offsets are NULL");
        static DevBuf<int64_t> scratch;   // library-owned, grown on demand
        static std::mutex mu;
        std::lock_guard<std::mutex> lk(mu);
        exclusive_scan_i32(counts, n, offsets, scratch, as_stream(stream));
        CI_CUDA(cudaStreamSynchronize(as_stream(stream)));
    });
}

ci_status ci_build_H(ci_problem *p, int32_t vtype, ci_matrix **out, void *stream) {
    return guard([&] {
        StreamScope scope(as_stream(stream));
        if (!p || !out) fail(CI_ERR_INVALID_ARG, "problem or out is NULL");
        *out = nullptr;
        std::unique_ptr<ci_matrix> m(new ci_matrix());
        build_matrix(&p->impl, vtype, &m->impl, as_stream(stream));
        CI_CUDA(cudaStreamSynchronize(as_stream(stream)));
        *out = m.release();
    });
}

ci_status ci_matrix_upper(const ci_matrix *m, ci_matrix **out, void *stream) {
    return guard([&] {
        StreamScope scope(as_stream(stream));
        if (!m || !out) fail(CI_ERR_INVALID_ARG, "matrix or out is NULL");
        *out = nullptr;
        std::unique_ptr<ci_matrix> u(new ci_matrix());
        upper_matrix(&m->impl, &u->impl, as_stream(stream));
        CI_CUDA(cudaStreamSynchronize(as_stream(stream)));
        *out = u.release();
    });
}

void ci_matrix_destroy(ci_matrix *m) {
    if (!m) return;
    HandleRelease hr;
    delete m;
}

ci_status ci_matrix_info(const ci_matrix *m, int64_t *dim, int64_t *nnz, int32_t *vtype) {
    return guard([&] {
        if (!m) fail(CI_ERR_INVALID_ARG, "matrix is NULL");
        if (dim) *dim = m->impl.dim;
        if (nnz) *nnz = m->impl.nnz;
        if (vtype) *vtype = m->impl.vtype;
    });
}

ci_status ci_matrix_export(const ci_matrix *m, int64_t *row_ptr, int32_t *col, void *val, float *row_scale,
                           void *stream) {
    return guard([&] {
        StreamScope scope(as_stream(stream));
        if (!m) fail(CI_ERR_INVALID_ARG, "matrix is NULL");
        const Matrix &M = m->impl;
        cudaStream_t s = as_stream(stream);
        size_t esz = M.vtype == CI_F64 ? 8 : (M.vtype == CI_F32 ? 4 : 2);
        copy_out(row_ptr, M.row_ptr.ptr, (M.dim + 1) * sizeof(int64_t), s);
        copy_out(col, M.col.ptr, M.nnz * sizeof(int32_t), s);
        copy_out(val, M.val.ptr, M.nnz * esz, s);
        if (M.vtype == CI_BF16_ROWSCALE) copy_out(row_scale, M.row_scale.ptr, M.dim * sizeof(float), s);
        CI_CUDA(cudaStreamSynchronize(s));
    });
}

ci_status ci_apply_H(const ci_matrix *m, const void *X, void *Y, int32_t nvec, void *stream) {
    return guard([&] {
        StreamScope scope(as_stream(stream));
        if (!m) fail(CI_ERR_INVALID_ARG, "matrix is NULL");
        apply_matrix(&m->impl, X, Y, nvec, as_stream(stream));
    });
}

}  // extern "C"
