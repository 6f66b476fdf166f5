// Kernel launch accounting and opt-in per-kernel timing with CUDA events recorded on the
// launching stream (used by the benchmark to time the dominant kernel inside a run).
#include <atomic>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace iim {

static std::atomic<long long> g_launches{0};

struct TraceRec {
    const char* name;
    cudaEvent_t a, b;
    double bytes, flops;
};
static thread_local bool t_prof = false;
static thread_local bool t_capture = false;
static thread_local std::vector<TraceRec> t_recs;
static thread_local std::vector<cudaEvent_t> t_pool;
static thread_local size_t t_pool_used = 0;

static cudaEvent_t pool_event() {
    if (t_pool_used == t_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        t_pool.push_back(e);
    }
    return t_pool[t_pool_used++];
}

void set_capture(bool on) { t_capture = on; }
bool profiling_active() { return t_prof; }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

KTrace::KTrace(const char* name, cudaStream_t s, double bytes, double flops) : active(false), stream(s), idx(0) {
    if (t_capture) return;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!t_prof) return;
    TraceRec r{name, pool_event(), pool_event(), bytes, flops};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    idx = (int)t_recs.size();
    t_recs.push_back(r);
    active = true;
}

KTrace::~KTrace() {
    if (active) cudaEventRecord(t_recs[idx].b, stream);
}

}  // namespace iim

using namespace iim;

extern "C" long long iim_launch_count(void) { return g_launches.load(); }

extern "C" iim_status iim_profile_begin(void) {
    t_recs.clear();
    t_pool_used = 0;
    t_prof = true;
    return IIM_OK;
}

extern "C" int iim_profile_end(iim_kernel_stat* out, int capacity) {
    t_prof = false;
    std::vector<iim_kernel_stat> agg;
    for (const TraceRec& r : t_recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
        size_t k = 0;
        for (; k < agg.size(); ++k)
            if (std::strcmp(agg[k].name, r.name) == 0) break;
        if (k == agg.size()) agg.push_back(iim_kernel_stat{r.name, 0, 0.0, 0.0, 0.0});
        agg[k].launches += 1;
        agg[k].ms += ms;
        agg[k].bytes += r.bytes;
        agg[k].flops += r.flops;
    }
    t_recs.clear();
    t_pool_used = 0;
    const int n = (int)agg.size();
    for (int k = 0; k < n && k < capacity && out; ++k) out[k] = agg[k];
    return n;
}
