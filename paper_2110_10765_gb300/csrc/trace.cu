// Kernel tracing (ci_trace_enable / ci_trace_read): CUDA events around every
// library launch, summed per kernel name when read.
#include <map>
#include <mutex>
#include <string>

#include "problem.cuh"

namespace ci {

namespace {
struct Pending {
    std::string name;
    cudaEvent_t a, b;
};
struct Stat {
    int64_t launches = 0;
    double ms = 0.0;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Pending *> g_pending;
std::map<std::string, Stat> g_stats;
std::vector<cudaEvent_t> g_free;   // recycled events (creating one per launch costs host time)

cudaEvent_t take_event() {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_free.empty()) {
            cudaEvent_t e = g_free.back();
            g_free.pop_back();
            return e;
        }
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
            Stat &s = g_stats[p->name];
            s.launches += 1;
            s.ms += ms;
        }
        g_free.push_back(p->a);
        g_free.push_back(p->b);
        delete p;
    }
    g_pending.clear();
    cudaGetLastError();
}
}  // namespace

bool trace_on() { return g_on; }

void trace_begin(const char *name, cudaStream_t s, void **token) {
    Pending *p = new Pending{name, take_event(), take_event()};
    if (!p->a || !p->b) {
        std::lock_guard<std::mutex> lk(g_mu);
        if (p->a) g_free.push_back(p->a);
        if (p->b) g_free.push_back(p->b);
        delete p;
        *token = nullptr;
        return;
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
        std::lock_guard<std::mutex> lk(ci::g_mu);
        ci::g_on = on != 0;
    });
}

ci_status ci_trace_read(ci_trace_entry *out, int32_t cap, int32_t *n, int32_t reset) {
    return ci::guard([&] {
        std::lock_guard<std::mutex> lk(ci::g_mu);
        ci::drain_locked();
        int32_t i = 0;
        for (auto &kv : ci::g_stats) {
            if (out && i < cap) {
                std::snprintf(out[i].name, sizeof(out[i].name), "%s", kv.first.c_str());
                out[i].launches = kv.second.launches;
                out[i].total_ms = kv.second.ms;
            }
            ++i;
        }
        if (n) *n = i;
        if (reset) ci::g_stats.clear();
    });
}

}  // extern "C"
