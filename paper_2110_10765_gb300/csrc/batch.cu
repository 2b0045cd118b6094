// Batched solves (ci_batch_*): many independent problems built in one
// grouped launch per build step and solved together by the engine.
#include <chrono>

#include "engine.cuh"

namespace ci {

struct Batch {
    std::vector<Problem *> probs;
    std::vector<int> k;
    ci_eig_opts opts{};
    int MB = 64;
    GroupCSR csr;
    DevBuf<double> Q, W;
    DevBuf<float> X, Y;
    Engine eng;
    bool ran = false;
    double build_s = 0, solve_s = 0;
    int steps = 0;
};

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void batch_run(Batch *b, cudaStream_t s) {
    const double t0 = now_s();
    const int n = (int)b->probs.size();
    for (Problem *p : b->probs) {
        enumerate_basis(p, s);
        if (p->dim <= (int64_t)b->MB + 2 * EB)
            fail(CI_ERR_INVALID_ARG, "batched solves need dimension > %d (got %lld)", b->MB + 2 * EB, (long long)p->dim);
    }
    count_group(b->probs, 0, &b->csr, s);
    fill_group(b->probs, &b->csr, s);
    CI_CUDA(cudaStreamSynchronize(s));
    const double t1 = now_s();
    const int64_t rows = b->csr.row_off.back();
    b->Q.alloc((size_t)rows * b->MB);
    b->W.alloc((size_t)rows * EB);
    b->X.alloc((size_t)rows * EB);
    b->Y.alloc((size_t)rows * EB);
    int64_t tiles = 0;
    for (Problem *p : b->probs) tiles += (p->dim + ETILE - 1) / ETILE;
    engine_create(&b->eng, n, (int)std::max<int64_t>(tiles, 1), b->MB, s);
    for (int i = 0; i < n; ++i) {
        const int64_t r0 = b->csr.row_off[i];
        SlotDev d{};
        d.dim = b->probs[i]->dim;
        d.rp = b->csr.row_ptr.ptr + r0;
        d.col = b->csr.col.ptr;
        d.val = (const float *)b->csr.val.ptr;
        d.Q = b->Q.ptr + r0 * b->MB;
        d.W = b->W.ptr + r0 * EB;
        d.X = b->X.ptr + r0 * EB;
        d.Y = b->Y.ptr + r0 * EB;
        d.k = b->k[i];
        d.max_iter = b->opts.max_iter;
        d.check_every = b->opts.check_every;
        d.tol = b->opts.tol;
        // start block from the problem itself (seed, size), not its slot, so a
        // problem gets the same result alone and in any mix
        const Problem *p = b->probs[i];
        d.seed = b->opts.seed ^ (p->tbme_seed * 0x9E3779B97F4A7C15ull + (uint64_t)p->dim);
        engine_set_slot(&b->eng, i, d);
    }
    engine_retile(&b->eng);
    engine_init_slots(&b->eng);
    int steps = engine_autotune(&b->eng);   // real steps, timed per launch shape
    while (true) {
        engine_step(&b->eng);
        ++steps;
        if (steps % 4 == 0 || steps >= b->opts.max_iter) {
            if (engine_running(&b->eng) == 0) break;
            if (steps >= b->opts.max_iter + 1) break;
        }
    }
    engine_true_residuals(&b->eng);
    b->steps = steps;
    const double t2 = now_s();
    b->build_s = t1 - t0;
    b->solve_s = t2 - t1;
    b->ran = true;
}

}  // namespace ci

struct ci_batch { ci::Batch impl; };

using namespace ci;

extern "C" {

ci_status ci_batch_create(ci_problem *const *probs, int32_t n, const int32_t *k, const ci_eig_opts *opts,
                          ci_batch **out) {
    return guard([&] {
        if (!out) fail(CI_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        if (!probs || n < 1) fail(CI_ERR_INVALID_ARG, "need at least one problem");
        std::unique_ptr<ci_batch> b(new ci_batch());
        Batch &B = b->impl;
        B.opts = opts ? *opts : ci_eig_opts{};
        if (B.opts.max_basis == 0) B.opts.max_basis = 64;
        if (B.opts.max_iter == 0) B.opts.max_iter = 400;
        if (B.opts.tol == 0.0) B.opts.tol = 1e-7;
        if (B.opts.seed == 0) B.opts.seed = 1;
        if (B.opts.check_every == 0) B.opts.check_every = 4;
        if (B.opts.block != 0 && B.opts.block != EB) fail(CI_ERR_INVALID_ARG, "batched solves use block size 8");
        B.MB = B.opts.max_basis;
        if (B.MB % EB || B.MB < 4 * EB || B.MB > EMBMAX)
            fail(CI_ERR_INVALID_ARG, "max_basis must be a multiple of 8 in 32..96 for batched solves");
        for (int i = 0; i < n; ++i) {
            if (!probs[i]) fail(CI_ERR_INVALID_ARG, "problem %d is NULL", i);
            const int ki = k ? k[i] : (B.opts.k ? B.opts.k : 5);
            if (ki < 1 || ki > EKMAX || 2 * (ki + EB) > B.MB)
                fail(CI_ERR_INVALID_ARG, "k[%d] = %d must be 1..%d with 2(k+8) <= max_basis", i, ki, EKMAX);
            B.probs.push_back(&probs[i]->impl);
            B.k.push_back(ki);
        }
        *out = b.release();
    });
}

ci_status ci_batch_run(ci_batch *b, void *stream) {
    return guard([&] {
        if (!b) fail(CI_ERR_INVALID_ARG, "batch is NULL");
        if (b->impl.ran) fail(CI_ERR_STATE, "batch already ran");
        StreamScope scope(reinterpret_cast<cudaStream_t>(stream));
        batch_run(&b->impl, reinterpret_cast<cudaStream_t>(stream));
    });
}

ci_status ci_batch_tuning(const ci_batch *b, int32_t *tile_ctas_per_sm, int32_t *spmm_ctas_per_sm,
                          double *best_step_ms) {
    return guard([&] {
        if (!b) fail(CI_ERR_INVALID_ARG, "batch is NULL");
        if (!b->impl.ran) fail(CI_ERR_STATE, "call ci_batch_run first");
        if (tile_ctas_per_sm) *tile_ctas_per_sm = b->impl.eng.tile_mult;
        if (spmm_ctas_per_sm) *spmm_ctas_per_sm = b->impl.eng.spmm_mult;
        if (best_step_ms) *best_step_ms = b->impl.eng.tuned_step_ms;
    });
}

ci_status ci_batch_result(const ci_batch *b, int32_t i, double *evals, ci_eig_info *info) {
    return guard([&] {
        if (!b) fail(CI_ERR_INVALID_ARG, "batch is NULL");
        const Batch &B = b->impl;
        if (!B.ran) fail(CI_ERR_STATE, "call ci_batch_run first");
        if (i < 0 || i >= (int)B.probs.size()) fail(CI_ERR_INVALID_ARG, "index %d out of range", i);
        double ev[EKMAX], est[EKMAX], tr[EKMAX];
        int it = 0, st = 0;
        engine_results(const_cast<Engine *>(&B.eng), i, ev, est, tr, &it, &st);
        const int k = B.k[i];
        if (evals)
            for (int j = 0; j < k; ++j) evals[j] = ev[j];
        if (info) {
            *info = ci_eig_info{};
            info->iterations = it;
            info->converged = st == S_CONV ? k : 0;
            info->basis_size = B.MB;
            for (int j = 0; j < k && j < 32; ++j) info->residual[j] = tr[j];
            info->seconds = B.solve_s;
            info->hnorm_est = 0.0;
        }
        if (st != S_CONV) fail(CI_ERR_NOT_CONVERGED, "problem %d did not converge in %d steps", i, it);
    });
}

ci_status ci_batch_stats(const ci_batch *b, double *build_s, double *solve_s, int32_t *steps, int64_t *nnz) {
    return guard([&] {
        if (!b) fail(CI_ERR_INVALID_ARG, "batch is NULL");
        if (build_s) *build_s = b->impl.build_s;
        if (solve_s) *solve_s = b->impl.solve_s;
        if (steps) *steps = b->impl.steps;
        if (nnz) *nnz = b->impl.csr.nnz;
    });
}

void ci_batch_destroy(ci_batch *b) {
    if (!b) return;
    HandleRelease hr;
    delete b;
}

}  // extern "C"
