// gp_prof.cu -- kernel launch counter and optional CUDA-event timing of the
// library's kernel groups (host code only).
//
// When profiling is enabled, every kernel group (tables, Gram, assembly,
// Cholesky, inverse, solve, packing, predict) is bracketed by two CUDA events
// recorded on the stream it is launched on; gp_profile_query() waits for the
// events and reports launches and total device milliseconds per group.
#include "gp_common.cuh"

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace {

std::atomic<long long> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;

struct Pending {
    std::string name;
    cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::map<std::string, std::pair<long long, double>> g_totals;
std::map<cudaStream_t, cudaEvent_t> g_open;  // stream -> start event of the open group
std::map<cudaStream_t, std::string> g_open_name;
std::vector<cudaEvent_t> g_free_events;

cudaEvent_t get_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void drain_locked() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        cudaEventElapsedTime(&ms, p.a, p.b);
        auto& t = g_totals[p.name];
        t.first += 1;
        t.second += ms;
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace

void gp_note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Switch the group timing off (returning its previous state) and back on:
// work that is captured into a graph is not timed.
int gp_prof_suspend() { return g_prof_on.exchange(0); }
void gp_prof_resume(int state) { g_prof_on.store(state); }

void gp_prof_begin(const char* name, cudaStream_t s) {
    if (!g_prof_on.load()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e = get_event();
    cudaEventRecord(e, s);
    g_open[s] = e;
    g_open_name[s] = name;
}

void gp_prof_end(const char* name, cudaStream_t s) {
    if (!g_prof_on.load()) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    auto it = g_open.find(s);
    if (it == g_open.end() || g_open_name[s] != name) return;
    cudaEvent_t b = get_event();
    cudaEventRecord(b, s);
    g_pending.push_back({name, it->second, b});
    g_open.erase(it);
}

extern "C" {

GPFAGP_API int64_t gp_kernel_launches(void) { return (int64_t)g_launches.load(); }

GPFAGP_API void gp_profile_enable(int on) { g_prof_on.store(on ? 1 : 0); }

GPFAGP_API void gp_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_locked();
    g_totals.clear();
}

GPFAGP_API int gp_profile_query(const char* name, int64_t* launches, double* total_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    drain_locked();
    auto it = g_totals.find(name ? name : "");
    if (it == g_totals.end()) {
        if (launches) *launches = 0;
        if (total_ms) *total_ms = 0.0;
        return GP_EINVAL;
    }
    if (launches) *launches = it->second.first;
    if (total_ms) *total_ms = it->second.second;
    return GP_OK;
}

}  // extern "C"
