// Per-stage counters and CUDA-event timing (see profile.h).
#include <mutex>
#include <vector>

#include "../../include/mdls.h"
#include "profile.h"

namespace mdls {
namespace {

struct Pending {
    int stage;
    cudaEvent_t a, b;
};

struct Profiler {
    std::mutex mu;
    bool timing = false;
    long long launches[ST_COUNT] = {};
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t open_ev[ST_COUNT] = {};
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

Profiler& prof() {
    static Profiler p;
    return p;
}

const char* kNames[ST_COUNT] = {"panel (beta, v; beta R^T v; update R)",
                                "compute W (Y^T Y, T, W = -Y T)",
                                "trailing update (YWT * C, R + YWTC)",
                                "Q accumulation (Q * WY^T, Q + QWY)",
                                "invert diagonal tiles",
                                "multiply with inverses",
                                "back substitution (right-hand side update)",
                                "other (copies, identity, zeroing, vector ops)",
                                "refinement (residuals, Q^T r, corrections)"};

}  // namespace

void stage_begin(int stage, cudaStream_t st) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.launches[stage] += 0;
    if (p.timing) {
        cudaEvent_t e = p.take();
        cudaEventRecord(e, st);
        p.open_ev[stage] = e;
    }
}

void stage_end(int stage, cudaStream_t st) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.launches[stage] += 1;
    if (p.timing && p.open_ev[stage]) {
        cudaEvent_t e = p.take();
        cudaEventRecord(e, st);
        p.pending.push_back({stage, p.open_ev[stage], e});
        p.open_ev[stage] = nullptr;
    }
}

}  // namespace mdls

using namespace mdls;

extern "C" {

void mdls_profile_enable(int on) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.timing = on != 0;
}

int mdls_profile_read(double* ms, int64_t* launches, int cap) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    double acc[ST_COUNT] = {};
    int rc = MDLS_OK;
    for (const Pending& q : p.pending) {
        float t = 0.f;
        if (cudaEventSynchronize(q.b) != cudaSuccess || cudaEventElapsedTime(&t, q.a, q.b) != cudaSuccess)
            rc = MDLS_ERR_CUDA;
        acc[q.stage] += t;
        p.pool.push_back(q.a);
        p.pool.push_back(q.b);
    }
    p.pending.clear();
    for (int s = 0; s < ST_COUNT && s < cap; ++s) {
        if (ms) ms[s] = acc[s];
        if (launches) launches[s] = p.launches[s];
        p.launches[s] = 0;
    }
    return rc == MDLS_OK ? ST_COUNT : rc;
}

}  // extern "C"

namespace mdls {
// Pauses event timing (launch counts continue) while a graph is captured,
// so that no timing events are recorded into the graph; returns the old state.
bool profiler_pause() {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    const bool old = p.timing;
    p.timing = false;
    return old;
}
void profiler_resume(bool on) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    p.timing = on;
}
}  // namespace mdls

extern "C" {

const char* mdls_stage_name(int stage) {
    if (stage < 0 || stage >= ST_COUNT) return "unknown stage";
    return kNames[stage];
}

}  // extern "C"
