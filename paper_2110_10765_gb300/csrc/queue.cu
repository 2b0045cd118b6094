// Solve queue with continuous batching (ci_queue_*, ci_submit, ci_poll,
// ci_cancel).  A worker thread owns the device loop: between two replays of
// the engine's step graph it harvests finished slots (FP64 residuals,
// results, memory released) and admits pending requests into free slots as
// long as their device memory fits the budget; admitted requests are built
// together (one launch per build step) and join the running ones at the
// next step, so requests that arrive while others run overlap with them.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "engine.cuh"

namespace ci {

static double qnow() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    std::vector<int32_t> spN, spm;
    std::vector<double> eps;
    std::vector<unsigned char> tabs[3];
    ci_problem_desc desc{};
    int k = 5;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int status = CI_NOT_READY;
    std::string error;
    bool cancelled = false;
    std::unique_ptr<ci_problem> prob;
    std::shared_ptr<GroupCSR> group;
    DevBuf<double> Q, W;
    DevBuf<float> X, Y;
    int slot = -1;
    size_t mem = 0;
    int64_t dim = 0, nnz = 0;
    int iterations = 0;
    double evals[EKMAX] = {0}, residual[EKMAX] = {0};
};

struct Queue {
    ci_queue_desc d{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> pending;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    std::vector<Request *> in_slot;
    uint64_t next_ticket = 1;
    Engine eng;
    std::thread worker;
    bool stop = false;
    size_t mem_used = 0;
    int64_t tiles_used = 0;
    int64_t steps = 0, admitted = 0, completed = 0;
    std::string fatal;

    void run();
    void admit();
    void harvest();
    void solve_small(Request *r);
};

// Device bytes a request holds while it runs.
static size_t request_bytes(const Problem *p, int64_t nnz, int MB) {
    const int64_t dim = p->dim;
    size_t b = (size_t)nnz * 8 + (size_t)(dim + 1) * 8 + (size_t)dim * 12;            // CSR + counts + row map
    b += (size_t)dim * ((size_t)MB * 8 + EB * 8 + 2 * EB * 4);                          // Q, W, X, Y
    const Connectivity<float> &c = p->c32;
    b += (size_t)(c.outer.total + c.outer4.total + c.l2.total + c.l4.total) * (sizeof(ConnEntry<float>) + 4);
    const size_t S = (size_t)p->S;
    b += (S * S * S * 4 + p->like_size * 2 + p->tr_size + S * S * 3) * sizeof(float);  // staged tables
    return b;
}

void Queue::harvest() {
    // slot states from the device (one small copy), then FP64 residuals and
    // results of the slots that finished
    std::vector<SlotDev> cur(eng.max_slots);
    CI_CUDA(cudaMemcpyAsync(cur.data(), eng.slots.ptr, sizeof(SlotDev) * eng.max_slots, cudaMemcpyDeviceToHost,
                            eng.stream));
    CI_CUDA(cudaStreamSynchronize(eng.stream));
    std::vector<int> done;
    for (int i = 0; i < eng.max_slots; ++i) {
        Request *r = in_slot[i];
        if (!r) continue;
        if (cur[i].state == S_CONV || cur[i].state == S_FAIL || r->cancelled) done.push_back(i);
    }
    if (done.empty()) return;
    engine_true_residuals(&eng);
    const double t = qnow();
    std::lock_guard<std::mutex> lk(mu);
    for (int i : done) {
        Request *r = in_slot[i];
        int st = 0, it = 0;
        double ev[EKMAX], est[EKMAX], tr[EKMAX];
        engine_results(&eng, i, ev, est, tr, &it, &st);
        for (int j = 0; j < r->k; ++j) { r->evals[j] = ev[j]; r->residual[j] = tr[j]; }
        r->iterations = it;
        r->t_done = t;
        if (r->cancelled) r->status = CI_ERR_CANCELLED;
        else r->status = st == S_CONV ? CI_OK : CI_ERR_NOT_CONVERGED;
        if (r->status == CI_ERR_NOT_CONVERGED) r->error = "did not converge";
        engine_free_slot(&eng, i);
        in_slot[i] = nullptr;
        mem_used -= r->mem;
        tiles_used -= (r->dim + ETILE - 1) / ETILE;
        r->Q.release(); r->W.release(); r->X.release(); r->Y.release();
        r->group.reset();
        r->prob.reset();
        ++completed;
    }
    engine_retile(&eng);
}

void Queue::admit() {
    std::vector<Request *> cand;
    {
        std::lock_guard<std::mutex> lk(mu);
        int free_slots = 0;
        for (Request *r : in_slot) free_slots += r == nullptr;
        while (!pending.empty() && (int)cand.size() < free_slots) {
            Request *r = pending.front();
            pending.pop_front();
            if (r->cancelled) { r->status = CI_ERR_CANCELLED; r->t_done = qnow(); continue; }
            cand.push_back(r);
        }
    }
    if (cand.empty()) return;
    // create and count the candidates together; spaces too small for the
    // engine's Krylov blocks are solved at once on the single-problem path
    std::vector<Request *> ok, small;
    for (Request *r : cand) {
        try {
            r->prob.reset(new ci_problem());
            problem_create(&r->desc, &r->prob->impl);
            enumerate_basis(&r->prob->impl, eng.stream);
            if (r->prob->impl.dim <= (int64_t)eng.MB + 2 * EB) small.push_back(r);
            else ok.push_back(r);
        } catch (const Error &e) {
            std::lock_guard<std::mutex> lk(mu);
            r->status = e.status; r->error = e.what(); r->t_done = qnow(); r->prob.reset();
        }
    }
    for (Request *r : small) solve_small(r);
    if (ok.empty()) return;
    std::vector<Problem *> ps;
    for (Request *r : ok) ps.push_back(&r->prob->impl);
    auto g = std::make_shared<GroupCSR>();
    count_group(ps, 0, g.get(), eng.stream);
    // requests that can never fit are refused; then the FIFO prefix that
    // fits the memory budget and the tile list is admitted, the rest waits
    std::vector<Request *> adm, wait;
    std::vector<Problem *> aps;
    size_t used = mem_used;
    int64_t tiles = tiles_used;
    bool blocked = false;
    for (size_t i = 0; i < ok.size(); ++i) {
        const size_t b = request_bytes(ps[i], g->nnz_of[i], eng.MB);
        const int64_t t = (ps[i]->dim + ETILE - 1) / ETILE;
        if (b > d.mem_budget || t > eng.max_tiles) {
            std::lock_guard<std::mutex> lk(mu);
            ok[i]->status = CI_ERR_CAPACITY;
            ok[i]->error = "request needs more device memory than the queue's budget";
            ok[i]->t_done = qnow();
            ok[i]->prob.reset();
            continue;
        }
        if (blocked || used + b > d.mem_budget || tiles + t > eng.max_tiles) {
            blocked = true;
            wait.push_back(ok[i]);
            continue;
        }
        ok[i]->mem = b;
        used += b;
        tiles += t;
        adm.push_back(ok[i]);
        aps.push_back(ps[i]);
    }
    if (!wait.empty()) {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = wait.size(); i-- > 0;) {
            wait[i]->prob.reset();
            pending.push_front(wait[i]);
        }
    }
    if (adm.empty()) return;
    if (adm.size() != ok.size()) {  // recount the admitted set as one group
        g = std::make_shared<GroupCSR>();
        count_group(aps, 0, g.get(), eng.stream);
    }
    ok = adm;
    ps = aps;
    fill_group(ps, g.get(), eng.stream);
    const double t = qnow();
    int slot = 0;
    for (size_t i = 0; i < ok.size(); ++i) {
        Request *r = ok[i];
        while (in_slot[slot]) ++slot;
        const int64_t dim = ps[i]->dim, r0 = g->row_off[i];
        r->Q.alloc((size_t)dim * eng.MB);
        r->W.alloc((size_t)dim * EB);
        r->X.alloc((size_t)dim * EB);
        r->Y.alloc((size_t)dim * EB);
        SlotDev sd{};
        sd.dim = dim;
        sd.rp = g->row_ptr.ptr + r0;
        sd.col = g->col.ptr;
        sd.val = (const float *)g->val.ptr;
        sd.Q = r->Q.ptr; sd.W = r->W.ptr; sd.X = r->X.ptr; sd.Y = r->Y.ptr;
        sd.k = r->k;
        sd.max_iter = d.max_iter;
        sd.check_every = 4;
        sd.tol = d.tol;
        sd.seed = 1ull ^ (r->desc.tbme_seed * 0x9E3779B97F4A7C15ull + (uint64_t)dim);
        engine_set_slot(&eng, slot, sd);
        std::lock_guard<std::mutex> lk(mu);
        r->group = g;
        r->slot = slot;
        r->dim = dim;
        r->nnz = g->nnz_of[i];
        r->t_admit = t;
        in_slot[slot] = r;
        mem_used += r->mem;
        tiles_used += (dim + ETILE - 1) / ETILE;
        ++admitted;
    }
    engine_retile(&eng);
    engine_init_slots(&eng);
}

// A request whose basis has at most MB + 2 EB states: FP32 H built alone
// and solved by the single-problem eigensolver (Rayleigh-Ritz on the whole
// space at this size) on the engine stream, between two engine steps.
void Queue::solve_small(Request *r) {
    const double t0 = qnow();
    try {
        Problem *p = &r->prob->impl;
        Matrix m;
        build_matrix(p, CI_F32, &m, eng.stream);
        ci_eig_opts o{};
        o.k = r->k;
        o.block = EB;
        o.max_basis = eng.MB;
        o.tol = d.tol;
        double ev[32] = {0};
        ci_eig_info inf{};
        lowest_eigs(&m, &o, ev, nullptr, &inf, eng.stream);
        std::lock_guard<std::mutex> lk(mu);
        for (int j = 0; j < r->k; ++j) { r->evals[j] = ev[j]; r->residual[j] = inf.residual[j]; }
        r->iterations = inf.iterations;
        r->dim = m.dim;
        r->nnz = m.nnz;
        r->t_admit = t0;
        r->t_done = qnow();
        r->status = CI_OK;
        ++admitted;
        ++completed;
    } catch (const Error &e) {
        std::lock_guard<std::mutex> lk(mu);
        r->status = e.status;
        r->error = e.what();
        r->t_done = qnow();
    }
    r->prob.reset();
}

void Queue::run() {
    try {
        CI_CUDA(cudaSetDevice(device));
        StreamScope scope(eng.stream);  // requests live on the engine stream
        int64_t since = 0;
        while (true) {
            {
                std::unique_lock<std::mutex> lk(mu);
                bool busy = false;
                for (Request *r : in_slot) busy |= r != nullptr;
                if (!busy && pending.empty()) {
                    if (stop) break;
                    cv.wait_for(lk, std::chrono::milliseconds(50));
                    continue;
                }
                if (stop) {  // cancel what is left
                    for (Request *r : pending) { r->status = CI_ERR_CANCELLED; r->t_done = qnow(); }
                    pending.clear();
                    for (Request *r : in_slot) if (r) r->cancelled = true;
                }
            }
            bool busy = false;
            for (Request *r : in_slot) busy |= r != nullptr;
            if (busy) {
                engine_step(&eng);
                ++steps;
                ++since;
            }
            if (!busy || since >= 2) {
                since = 0;
                if (busy) harvest();
                admit();
            }
        }
    } catch (const std::exception &e) {
        std::lock_guard<std::mutex> lk(mu);
        fatal = e.what();
        for (auto &kv : all)
            if (kv.second->status == CI_NOT_READY) { kv.second->status = CI_ERR_INTERNAL; kv.second->error = fatal; }
    }
}

}  // namespace ci

struct ci_queue { ci::Queue impl; };

using namespace ci;

extern "C" {

ci_status ci_queue_create(const ci_queue_desc *desc, ci_queue **out) {
    return guard([&] {
        if (!out) fail(CI_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        std::unique_ptr<ci_queue> q(new ci_queue());
        Queue &Q = q->impl;
        Q.d = desc ? *desc : ci_queue_desc{};
        if (Q.d.max_slots == 0) Q.d.max_slots = 256;
        if (Q.d.max_basis == 0) Q.d.max_basis = 64;
        if (Q.d.max_iter == 0) Q.d.max_iter = 400;
        if (Q.d.tol == 0.0) Q.d.tol = 1e-7;
        if (Q.d.max_slots < 1 || Q.d.max_slots > 4096) fail(CI_ERR_INVALID_ARG, "max_slots must be 1..4096");
        CI_CUDA(cudaGetDevice(&Q.device));
        if (Q.d.mem_budget == 0) {
            size_t fr = 0, tot = 0;
            CI_CUDA(cudaMemGetInfo(&fr, &tot));
            Q.d.mem_budget = fr / 10 * 7;
        }
        const int max_tiles = Q.d.max_tiles ? Q.d.max_tiles : 65536;
        engine_create(&Q.eng, Q.d.max_slots, max_tiles, Q.d.max_basis, nullptr);
        Q.in_slot.assign(Q.d.max_slots, nullptr);
        Q.worker = std::thread([&Q] { Q.run(); });
        *out = q.release();
    });
}

ci_status ci_submit(ci_queue *q, const ci_request *req, uint64_t *ticket) {
    return guard([&] {
        if (!q || !req || !ticket) fail(CI_ERR_INVALID_ARG, "queue, request and ticket are required");
        Queue &Q = q->impl;
        const ci_problem_desc &d = req->desc;
        if (d.n_sp < 1 || d.n_sp > 64 * kMaxWords || !d.sp_N || !d.sp_twom || !d.sp_energy)
            fail(CI_ERR_INVALID_ARG, "bad s.p. table");
        if (req->k < 1 || req->k > EKMAX || 2 * (req->k + EB) > Q.d.max_basis)
            fail(CI_ERR_INVALID_ARG, "k must be 1..%d with 2(k+8) <= max_basis", EKMAX);
        std::unique_ptr<Request> r(new Request());
        r->spN.assign(d.sp_N, d.sp_N + d.n_sp);
        r->spm.assign(d.sp_twom, d.sp_twom + d.n_sp);
        r->eps.assign(d.sp_energy, d.sp_energy + d.n_sp);
        r->desc = d;
        r->desc.sp_N = r->spN.data();
        r->desc.sp_twom = r->spm.data();
        r->desc.sp_energy = r->eps.data();
        if (d.tbme_source == CI_TBME_TABLES) {
            const size_t esz = d.tbme_dtype == CI_F64 ? 8 : 4;
            const size_t bytes = esz * (size_t)d.n_sp * d.n_sp * d.n_sp * d.n_sp;
            const void *src[3] = {d.v_pp, d.v_nn, d.v_pn};
            for (int c = 0; c < 3; ++c) {
                if (!src[c]) fail(CI_ERR_INVALID_ARG, "missing TBME table");
                r->tabs[c].resize(bytes);
                CI_CUDA(cudaMemcpy(r->tabs[c].data(), src[c], bytes, cudaMemcpyDefault));
            }
            r->desc.v_pp = r->tabs[0].data();
            r->desc.v_nn = r->tabs[1].data();
            r->desc.v_pn = r->tabs[2].data();
        }
        r->k = req->k;
        r->t_submit = qnow();
        std::lock_guard<std::mutex> lk(Q.mu);
        if (Q.stop) fail(CI_ERR_STATE, "queue is shutting down");
        if (!Q.fatal.empty()) fail(CI_ERR_INTERNAL, "queue stopped: %s", Q.fatal.c_str());
        r->ticket = Q.next_ticket++;
        *ticket = r->ticket;
        Q.pending.push_back(r.get());
        Q.all[r->ticket] = std::move(r);
        Q.cv.notify_all();
    });
}

ci_status ci_poll(ci_queue *q, uint64_t ticket, ci_result *res) {
    ci_status st = CI_OK;
    ci_status g = guard([&] {
        if (!q) fail(CI_ERR_INVALID_ARG, "queue is NULL");
        Queue &Q = q->impl;
        std::lock_guard<std::mutex> lk(Q.mu);
        auto it = Q.all.find(ticket);
        if (it == Q.all.end()) fail(CI_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
        Request *r = it->second.get();
        if (res) {
            *res = ci_result{};
            res->status = r->status;
            res->k = r->k;
            for (int j = 0; j < r->k; ++j) { res->evals[j] = r->evals[j]; res->residual[j] = r->residual[j]; }
            res->iterations = r->iterations;
            res->dim = r->dim;
            res->nnz = r->nnz;
            res->t_submit = r->t_submit;
            res->t_admit = r->t_admit;
            res->t_done = r->t_done;
            res->latency_s = r->status == CI_NOT_READY ? 0.0 : r->t_done - r->t_submit;
        }
        st = (ci_status)r->status;
        if (r->status != CI_OK && r->status != CI_NOT_READY) set_last_error(r->error);
    });
    return g != CI_OK ? g : st;
}

ci_status ci_cancel(ci_queue *q, uint64_t ticket) {
    return guard([&] {
        if (!q) fail(CI_ERR_INVALID_ARG, "queue is NULL");
        Queue &Q = q->impl;
        std::lock_guard<std::mutex> lk(Q.mu);
        auto it = Q.all.find(ticket);
        if (it == Q.all.end()) fail(CI_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
        if (it->second->status == CI_NOT_READY) it->second->cancelled = true;
    });
}

ci_status ci_queue_stats(ci_queue *q, int64_t *submitted, int64_t *admitted, int64_t *completed, int64_t *steps,
                         size_t *mem_used) {
    return guard([&] {
        if (!q) fail(CI_ERR_INVALID_ARG, "queue is NULL");
        Queue &Q = q->impl;
        std::lock_guard<std::mutex> lk(Q.mu);
        if (submitted) *submitted = (int64_t)Q.all.size();
        if (admitted) *admitted = Q.admitted;
        if (completed) *completed = Q.completed;
        if (steps) *steps = Q.steps;
        if (mem_used) *mem_used = Q.mem_used;
    });
}

void ci_queue_destroy(ci_queue *q) {
    if (!q) return;
    {
        std::lock_guard<std::mutex> lk(q->impl.mu);
        q->impl.stop = true;
        q->impl.cv.notify_all();
    }
    if (q->impl.worker.joinable()) q->impl.worker.join();
    HandleRelease hr;
    delete q;
}

}  // extern "C"
