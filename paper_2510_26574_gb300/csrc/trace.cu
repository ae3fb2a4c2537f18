// Tracing: per-stage CUDA-event timing of the library's own launches.
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "trace.cuh"

namespace kevd {

namespace {
// Open and closed intervals keyed by a handle that is never reused, so that
// host threads driving different streams can trace concurrently: a flush only
// consumes the intervals whose end has been recorded.
struct Pending {
    int stage;
    bool ended;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::map<int, Pending> g_pending;
int g_next = 0;
std::vector<cudaEvent_t> g_pool;
double g_ms[kNumStages];
long long g_launches[kNumStages];

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

int trace_begin(int stage, cudaStream_t s) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_on) return -1;
    Pending p{stage, false, take_event(), take_event()};
    if (!p.a || !p.b) return -1;
    cudaEventRecord(p.a, s);
    const int h = g_next;
    g_next = (g_next + 1) & 0x3fffffff;
    g_pending[h] = p;
    return h;
}

void trace_end(int h, cudaStream_t s) {
    if (h < 0) return;
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_pending.find(h);
    if (it == g_pending.end() || it->second.ended) return;
    cudaEventRecord(it->second.b, s);
    it->second.ended = true;
}

void trace_flush() {
    std::lock_guard<std::mutex> g(g_mu);
    for (auto it = g_pending.begin(); it != g_pending.end();) {
        if (!it->second.ended) {
            ++it;
            continue;
        }
        float ms = 0.f;
        const Pending& p = it->second;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.stage] += ms;
            g_launches[p.stage] += 1;
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
        it = g_pending.erase(it);
    }
}

}  // namespace kevd

using namespace kevd;

extern "C" int kevd_trace_enable(int on) {
    std::lock_guard<std::mutex> g(g_mu);
    const int prev = g_on;
    g_on = on != 0;
    return prev;
}

extern "C" void kevd_trace_reset(void) {
    std::lock_guard<std::mutex> g(g_mu);
    for (int i = 0; i < kNumStages; ++i) {
        g_ms[i] = 0.0;
        g_launches[i] = 0;
    }
}

extern "C" int kevd_trace_read(double* ms, int64_t* launches, int n) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!ms || !launches || n < 1) return KEVD_EINVAL;
    for (int i = 0; i < n && i < kNumStages; ++i) {
        ms[i] = g_ms[i];
        launches[i] = g_launches[i];
    }
    return KEVD_OK;
}
