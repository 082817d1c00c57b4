// Launch tracing: every kernel launch of the library bumps a counter; with timing
// enabled, the pair-sweep kernels are bracketed by CUDA events recorded on their
// launch stream, so a caller can read the average device duration of each kind
// over any region of its own program.
#include <atomic>
#include <mutex>
#include <vector>

#include "vpm_internal.h"

namespace vpm {

namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_timing{0};
std::mutex g_tmu;
struct Pair {
    cudaEvent_t a, b;
    int kind;
};
std::vector<Pair> g_pairs;       // recorded, not yet read
std::vector<cudaEvent_t> g_pool;  // free events
long long g_kind_launches[TRACE_KINDS];
double g_kind_ms[TRACE_KINDS];

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void drain_locked()
{
    for (auto& p : g_pairs) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_kind_launches[p.kind] += 1;
            g_kind_ms[p.kind] += ms;
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pairs.clear();
}
}  // namespace

void trace_launch(int count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

TraceScope::TraceScope(int kind, cudaStream_t st) : kind_(kind), st_(st)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_timing.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    a_ = take_event();
    b_ = take_event();
    if (a_ && b_) cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
}

TraceScope::~TraceScope()
{
    if (!a_ || !b_) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    cudaEventRecord(static_cast<cudaEvent_t>(b_), st_);
    g_pairs.push_back(Pair{static_cast<cudaEvent_t>(a_), static_cast<cudaEvent_t>(b_), kind_});
}

}  // namespace vpm

using namespace vpm;

extern "C" {

vpm_status vpm_trace_enable(int timing)
{
    g_timing.store(timing ? 1 : 0);
    return VPM_OK;
}

vpm_status vpm_trace_reset(void)
{
    std::lock_guard<std::mutex> lk(g_tmu);
    drain_locked();
    g_launches.store(0);
    for (int k = 0; k < TRACE_KINDS; ++k) g_kind_launches[k] = 0, g_kind_ms[k] = 0.0;
    return VPM_OK;
}

vpm_status vpm_trace_read(int kind, int64_t* launches, double* total_ms)
{
    if (kind < 0 || kind >= TRACE_KINDS || !launches || !total_ms) return VPM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tmu);
    drain_locked();
    if (kind == VPM_TRACE_ALL) {
        *launches = g_launches.load();
        double t = 0.0;
        for (int k = 1; k < TRACE_KINDS; ++k) t += g_kind_ms[k];
        *total_ms = t;
    } else {
        *launches = g_kind_launches[kind];
        *total_ms = g_kind_ms[kind];
    }
    return VPM_OK;
}

}  // extern "C"
