// Expectation values of two-body operators (Fig. 1, observables step; Fig. 2's
// element evaluation without the store; Sec. 2.4, Eq. 2):
//   a[k][v] = sum_ij X[i][v] (O_k)_ij X[j][v]
// for m operators O_k and n <= 8 vectors.  The elements of O_k are evaluated
// on the fly by the row kernels of the Hamiltonian build (same connectivity,
// the operator's tables) and multiplied into X at once; no operator is
// stored.  Each block leaves a partial of the n sums, the host adds them in
// block order (deterministic).
#include <cstring>

#include "problem.cuh"

namespace ci {

__global__ void k_pad8(int64_t dim, int n, const double *__restrict__ X, double *__restrict__ X8) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * 8; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t >> 3;
        const int q = (int)(t & 7);
        X8[t] = q < n ? X[i * n + q] : 0.0;
    }
}

void observables(Problem *P, const uint64_t *seeds, int m, const double *X, int n, double *a, cudaStream_t s) {
    if (!seeds || !a) fail(CI_ERR_INVALID_ARG, "op_seeds and a are required");
    if (m < 1 || m > 4096) fail(CI_ERR_INVALID_ARG, "m must be 1..4096 (got %d)", m);
    if (n < 1 || n > 8) fail(CI_ERR_INVALID_ARG, "n must be 1..8 (got %d)", n);
    enumerate_basis(P, s);
    if (P->dim > 0 && (!X || !is_device_pointer(X))) fail(CI_ERR_INVALID_ARG, "X must be a device pointer");
    std::memset(a, 0, sizeof(double) * (size_t)m * n);
    if (P->dim == 0) return;
    species_filter<double>(P, s);
    Connectivity<double> &c = P->conn<double>();
    const int64_t dim = P->dim;
    DevBuf<double> X8((size_t)dim * 8);
    launch("k_pad8", k_pad8, grid_for(dim * 8, 256), 256, 0, s, dim, n, X, X8.ptr);
    DevBuf<double> zero_eps((size_t)P->S);
    CI_CUDA(cudaMemsetAsync(zero_eps.ptr, 0, sizeof(double) * P->S, s));
    DevBuf<ConnEntry<double>> ents(c.outer.ent_buf->n);
    const int nblk_max = sm_count() * 8;
    DevBuf<double> part((size_t)m * nblk_max * 8);
    std::vector<int> nblk(m, 0);
    for (int k = 0; k < m; ++k) {
        Tables<double> t;
        stage_operator_tables<double>(P, seeds[k], t, zero_eps.ptr, s);
        operator_entries<double>(P, t, ents.ptr, s);
        nblk[k] = observable_apply<double>(P, t, ents.ptr, X8.ptr, part.ptr + (size_t)k * nblk_max * 8, s);
        if (nblk[k] > nblk_max) fail(CI_ERR_INTERNAL, "observable grid above its partial buffer");
    }
    std::vector<double> h((size_t)m * nblk_max * 8);
    CI_CUDA(cudaMemcpyAsync(h.data(), part.ptr, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    CI_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < m; ++k)
        for (int v = 0; v < n; ++v) {
            double t = 0.0;
            for (int b = 0; b < nblk[k]; ++b) t += h[((size_t)k * nblk_max + b) * 8 + v];
            a[(size_t)k * n + v] = t;
        }
}

}  // namespace ci

extern "C" ci_status ci_observables(ci_problem *p, const uint64_t *op_seeds, int32_t m, const double *X, int32_t n,
                                    double *a, void *stream) {
    return ci::guard([&] {
        if (!p) ci::fail(CI_ERR_INVALID_ARG, "problem is NULL");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ci::StreamScope scope(s);
        ci::observables(&p->impl, op_seeds, m, X, n, a, s);
    });
}
