// Expectation values and transition elements of two-body operators (Fig. 1,
// observables step; Fig. 2's element evaluation without the store; Sec. 2.4,
// Eq. 2):
//   a[k][v] = sum_ij X[i][v] (O_k)_ij Y[j][v]
// for m operators O_k and n <= 16 vector pairs (Y = X gives the expectation
// values).  The elements of O_k are evaluated on the fly by the row kernels
// of the Hamiltonian build (same connectivity, the operator's tables) and
// multiplied into Y at once; no operator is stored.  Vectors go through the
// row kernel eight at a time.  Each block leaves a partial of its eight sums,
// the host adds them in block order (deterministic).
#include <algorithm>
#include <cstring>

#include "problem.cuh"

namespace ci {

// X8[i][q] = X[i][g + q] for g + q < n, else 0 (columns g..g+7 of X [dim][n]).
__global__ void k_pad8(int64_t dim, int n, int g, const double *__restrict__ X, double *__restrict__ X8) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * 8; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t >> 3;
        const int q = g + (int)(t & 7);
        X8[t] = q < n ? X[i * n + q] : 0.0;
    }
}

void observables(Problem *P, const uint64_t *seeds, int m, const double *X, const double *Y, int n, double *a,
                 cudaStream_t s) {
    if (!seeds || !a) fail(CI_ERR_INVALID_ARG, "op_seeds and a are required");
    if (m < 1 || m > 4096) fail(CI_ERR_INVALID_ARG, "m must be 1..4096 (got %d)", m);
    if (n < 1 || n > 16) fail(CI_ERR_INVALID_ARG, "n must be 1..16 (got %d)", n);
    enumerate_basis(P, s);
    if (P->dim > 0 && (!X || !is_device_pointer(X))) fail(CI_ERR_INVALID_ARG, "X must be a device pointer");
    if (P->dim > 0 && Y && !is_device_pointer(Y)) fail(CI_ERR_INVALID_ARG, "Y must be a device pointer or NULL");
    std::memset(a, 0, sizeof(double) * (size_t)m * n);
    if (P->dim == 0) return;
    const bool same = !Y || Y == X;
    species_filter<double>(P, s);
    Connectivity<double> &c = P->conn<double>();
    const int64_t dim = P->dim;
    const int ng = (n + 7) / 8;
    DevBuf<double> L8((size_t)dim * 8 * ng), R8(same ? 0 : (size_t)dim * 8 * ng);
    for (int g = 0; g < ng; ++g) {
        launch("k_pad8", k_pad8, grid_for(dim * 8, 256), 256, 0, s, dim, n, 8 * g, X, L8.ptr + (size_t)g * dim * 8);
        if (!same)
            launch("k_pad8", k_pad8, grid_for(dim * 8, 256), 256, 0, s, dim, n, 8 * g, Y,
                   R8.ptr + (size_t)g * dim * 8);
    }
    const double *right = same ? L8.ptr : R8.ptr;
    DevBuf<double> zero_eps((size_t)P->S);
    CI_CUDA(cudaMemsetAsync(zero_eps.ptr, 0, sizeof(double) * P->S, s));
    DevBuf<ConnEntry<double>> ents(c.outer.ent_buf->n);
    const int nblk_max = sm_count() * 8;
    // operators in chunks: one partial array per (operator, group) of a chunk
    constexpr int kChunk = 64;
    const size_t slots = (size_t)std::min(m, kChunk) * ng;
    DevBuf<double> part(slots * nblk_max * 8);
    std::vector<double> h(slots * nblk_max * 8);
    for (int k0 = 0; k0 < m; k0 += kChunk) {
        const int kn = std::min(kChunk, m - k0);
        std::vector<int> nblk((size_t)kn * ng, 0);
        for (int kk = 0; kk < kn; ++kk) {
            Tables<double> t;
            stage_operator_tables<double>(P, seeds[k0 + kk], t, zero_eps.ptr, s);
            operator_entries<double>(P, t, ents.ptr, s);
            for (int g = 0; g < ng; ++g) {
                const size_t sl = (size_t)kk * ng + g;
                nblk[sl] = observable_apply<double>(P, t, ents.ptr, L8.ptr + (size_t)g * dim * 8,
                                                    right + (size_t)g * dim * 8, part.ptr + sl * nblk_max * 8, s);
                if (nblk[sl] > nblk_max) fail(CI_ERR_INTERNAL, "observable grid above its partial buffer");
            }
        }
        const size_t used = (size_t)kn * ng * nblk_max * 8;
        CI_CUDA(cudaMemcpyAsync(h.data(), part.ptr, sizeof(double) * used, cudaMemcpyDeviceToHost, s));
        CI_CUDA(cudaStreamSynchronize(s));
        for (int kk = 0; kk < kn; ++kk)
            for (int v = 0; v < n; ++v) {
                const size_t sl = (size_t)kk * ng + v / 8;
                double t = 0.0;
                for (int b = 0; b < nblk[sl]; ++b) t += h[(sl * nblk_max + b) * 8 + v % 8];
                a[(size_t)(k0 + kk) * n + v] = t;
            }
    }
}

}  // namespace ci

extern "C" ci_status ci_observables(ci_problem *p, const uint64_t *op_seeds, int32_t m, const double *X,
                                    const double *Y, int32_t n, double *a, void *stream) {
    return ci::guard([&] {
        if (!p) ci::fail(CI_ERR_INVALID_ARG, "problem is NULL");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        ci::StreamScope scope(s);
        ci::observables(&p->impl, op_seeds, m, X, Y, n, a, s);
    });
}
