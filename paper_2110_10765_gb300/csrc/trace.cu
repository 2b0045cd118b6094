// Kernel tracing (ci_trace_enable / ci_trace_read): every library launch is
// counted per kernel name, and CUDA events on the launch stream bracket
// either every launch (mode 1) or one launch in `mode` of each kernel (mode
// >= 2, sampled: the per-launch mean comes from the timed launches, the
// total is that mean times the launch count).  Sampling keeps the host cost
// of the events out of launch-bound loops.
#include <map>
#include <mutex>
#include <string>

#include "problem.cuh"

namespace ci {

namespace {
struct Stat {
    int64_t launches = 0;   // every launch
    int64_t timed = 0;      // launches with events
    double ms = 0.0;        // their summed durations
};
struct Pending {
    const char *name;       // the launch's kernel name (a string literal)
    cudaEvent_t a, b;
};
std::mutex g_mu;
int g_mode = 0;
std::vector<Pending *> g_pending;   // launches whose closing event is recorded
std::map<std::string, Stat> g_stats;
std::vector<cudaEvent_t> g_free;   // recycled events (creating one per launch costs host time)

cudaEvent_t take_event_locked() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void drain_locked() {
    for (Pending *p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p->b) == cudaSuccess && cudaEventElapsedTime(&ms, p->a, p->b) == cudaSuccess) {
            Stat &st = g_stats[p->name];
            st.timed += 1;
            st.ms += ms;
        }
        g_free.push_back(p->a);
        g_free.push_back(p->b);
        delete p;
    }
    g_pending.clear();
    cudaGetLastError();
}
}  // namespace

bool trace_on() { return g_mode != 0; }

void trace_begin(const char *name, cudaStream_t s, void **token) {
    *token = nullptr;
    Pending *p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_mode) return;
        Stat &st = g_stats[name];
        st.launches += 1;
        if (g_mode > 1 && (st.launches - 1) % g_mode != 0) return;   // counted, not timed
        p = new Pending{name, take_event_locked(), take_event_locked()};
        if (!p->a || !p->b) {
            if (p->a) g_free.push_back(p->a);
            if (p->b) g_free.push_back(p->b);
            delete p;
            return;
        }
    }
    cudaEventRecord(p->a, s);
    *token = p;
}

void trace_end(void *token, cudaStream_t s) {
    Pending *p = (Pending *)token;
    cudaEventRecord(p->b, s);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back(p);
    if (g_pending.size() > 4096) drain_locked();
}

}  // namespace ci

extern "C" {

ci_status ci_trace_enable(int32_t on) {
    return ci::guard([&] {
        if (on < 0) ci::fail(CI_ERR_INVALID_ARG, "trace mode must be >= 0 (got %d)", on);
        std::lock_guard<std::mutex> lk(ci::g_mu);
        ci::g_mode = on;
    });
}

ci_status ci_trace_read(ci_trace_entry *out, int32_t cap, int32_t *n, int32_t reset) {
    return ci::guard([&] {
        std::lock_guard<std::mutex> lk(ci::g_mu);
        ci::drain_locked();
        int32_t i = 0;
        for (auto &kv : ci::g_stats) {
            if (out && i < cap) {
                const ci::Stat &st = kv.second;
                std::snprintf(out[i].name, sizeof(out[i].name), "%s", kv.first.c_str());
                out[i].launches = st.launches;
                out[i].total_ms = st.timed ? st.ms * (double)st.launches / (double)st.timed : 0.0;
            }
            ++i;
        }
        if (n) *n = i;
        if (reset) ci::g_stats.clear();
    });
}

}  // extern "C"
