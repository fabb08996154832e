// profile.cu -- launch counter and optional per-stage CUDA-event timing.
//
// Timing is off unless ibpme_profile() enables a stage mask; then every
// enabled stage records an event pair on the stream it runs on, and
// ibpme_profile_read() synchronises, accumulates the elapsed times and
// returns per-stage totals and counts.
#include "common.cuh"

#include <atomic>
#include <mutex>
#include <vector>

namespace ibp {

namespace {

std::atomic<long long> g_launches{0};

struct Rec {
    int stage;
    cudaEvent_t a, b;
};

struct Profiler {
    std::mutex mu;
    unsigned mask = 0;
    std::vector<Rec> recs;
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
                                     "fft_forward64", "scale64", "fft_inverse64", "gather64"};

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfScope::ProfScope(int st, cudaStream_t strm) : stage(st), s(strm), on(false) {
    Profiler& p = prof();
    if (!(p.mask & (1u << st))) return;
    std::lock_guard<std::mutex> lk(p.mu);
    Rec r{st, p.take(), p.take()};
    IBP_CUDA(cudaEventRecord(r.a, s));
    p.recs.push_back(r);
    on = true;
}

ProfScope::~ProfScope() {
    if (!on) return;
    Profiler& p = prof();
    std::lock_guard<std::mutex> lk(p.mu);
    for (auto it = p.recs.rbegin(); it != p.recs.rend(); ++it)
        if (it->stage == stage) {
            cudaEventRecord(it->b, s);
            break;
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
