// profile.cu -- launch counter and optional per-stage CUDA-event timing.
//
// Timing is off unless ibpme_profile() enables a stage mask; then every
// enabled stage records an event pair on the stream it runs on, and
// ibpme_profile_read() synchronises, accumulates the elapsed times and
// returns per-stage totals and counts.
#include "common.cuh"

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

namespace ibp {

namespace {

std::atomic<long long> g_launches{0};

struct Rec {
    int stage;
    cudaEvent_t a, b;
    int gid;   // -1: ordinary launch; >= 0: event nodes of captured graph gid
};

struct Profiler {
    std::mutex mu;
    unsigned mask = 0;
    int capturing = -1;            // graph id being captured, -1 if none
    std::vector<Rec> recs;
    std::vector<Rec> graph_recs;   // event pairs owned by captured graphs
    std::vector<cudaEvent_t> pool;
    double total[ST_COUNT] = {};
    long long count[ST_COUNT] = {};

    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        IBP_CUDA(cudaEventCreate(&e));
        return e;
    }
    void drain() {   // caller holds mu; the events have completed
        for (const Rec& r : recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                total[r.stage] += ms;
                count[r.stage] += 1;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
    }
};

Profiler& prof() {
    static Profiler p;
    return p;
}

const char* kStageNames[ST_COUNT] = {"near_build", "near_apply", "spread", "fft_forward", "scale",
                                     "fft_inverse", "gather", "krylov", "bodies", "spread64",
                                     "fft_forward64", "scale64", "fft_inverse64", "gather64", "near_apply32",
                                     "near_field", "rpy_near"};

}  // namespace

void count_launch(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

ProfScope::ProfScope(int st, cudaStream_t strm) : stage(st), s(strm), on(false) {
    Profiler& p = prof();
    if (!(p.mask & (1u << st))) return;
    std::lock_guard<std::mutex> lk(p.mu);
    Rec r{st, p.take(), p.take(), p.capturing};
    // inside a stream capture an ordinary record only becomes a graph edge; an
    // external record becomes an event node that every replay re-records
    IBP_CUDA(cudaEventRecordWithFlags(r.a, s, r.gid >= 0 ? cudaEventRecordExternal : cudaEventRecordDefault));
    (r.gid >= 0 ? p.graph_recs : p.recs).push_back(r);
    on = true;
}

ProfScope::~ProfScope() {
    if (!on) return;
    Profiler& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    std::vector<Rec>& v = p.capturing >= 0 ? p.graph_recs : p.recs;
    for (auto it = v.rbegin(); it != v.rend(); ++it)
        if (it->stage == stage) {
            cudaEventRecordWithFlags(it->b, s, it->gid >= 0 ? cudaEventRecordExternal : cudaEventRecordDefault);
            break;
        }
}

unsigned prof_mask() {
    Profiler& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    return p.mask;
}

void prof_capture_begin(int gid) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    // a re-capture replaces the graph's previous event nodes
    for (auto it = p.graph_recs.begin(); it != p.graph_recs.end();) {
        if (it->gid == gid) {
            p.pool.push_back(it->a);
            p.pool.push_back(it->b);
            it = p.graph_recs.erase(it);
        } else {
            ++it;
        }
    }
    p.capturing = gid;
}

void prof_capture_end() {
    Profiler& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    p.capturing = -1;
}

void prof_graph_collect(int gid) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    for (const Rec& r : p.graph_recs) {
        if (r.gid != gid || !(p.mask & (1u << r.stage))) continue;
        float ms = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e == cudaSuccess) {
            p.total[r.stage] += ms;
            p.count[r.stage] += 1;
        } else {
            cudaGetLastError();   // a failed query must not surface as a later launch error
            if (std::getenv("IBPME_VERBOSE"))
                std::fprintf(stderr, "[ibpme] graph event timing failed for stage %d: %s\n", r.stage,
                             cudaGetErrorString(e));
        }
    }
}

}  // namespace ibp

using namespace ibp;

IBP_API long long ibpme_kernel_launches(void) { return g_launches.load(); }

IBP_API ibpme_status ibpme_profile(unsigned stage_mask) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    p.mask = stage_mask;
    for (int i = 0; i < ST_COUNT; ++i) {
        p.total[i] = 0.0;
        p.count[i] = 0;
    }
    if (!p.recs.empty()) {
        cudaDeviceSynchronize();
        p.drain();
        for (int i = 0; i < ST_COUNT; ++i) {
            p.total[i] = 0.0;
            p.count[i] = 0;
        }
    }
    return IBPME_OK;
}

IBP_API ibpme_status ibpme_profile_read(int max_stages, double* total_ms, long long* launches) {
    Profiler& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    if (!p.recs.empty()) {
        if (cudaDeviceSynchronize() != cudaSuccess) {
            set_error("cudaDeviceSynchronize failed while reading the profile");
            return IBPME_ERR_CUDA;
        }
        p.drain();
    }
    for (int i = 0; i < max_stages && i < ST_COUNT; ++i) {
        if (total_ms) total_ms[i] = p.total[i];
        if (launches) launches[i] = p.count[i];
    }
    return IBPME_OK;
}

IBP_API const char* ibpme_stage_name(int stage) {
    return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : "";
}
