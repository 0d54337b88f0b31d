// Launch counting and per-stage CUDA-event timing.
#include <atomic>

#include "grouped.h"
#include "prof.h"

namespace mfwq {

thread_local Profiler* g_prof = nullptr;
thread_local Recorder* g_rec = nullptr;
std::atomic<long long> g_launches{0};
namespace {
thread_local cudaEvent_t t_begin = nullptr;
thread_local bool t_open = false;
}  // namespace

static cudaEvent_t take_event(Profiler* p) {
    if (!p->free_events.empty()) {
        cudaEvent_t e = p->free_events.back();
        p->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void launch_begin(int tag, cudaStream_t s) {
    (void)tag;
    if (g_rec) return;  // recording: nothing is launched
    g_launches.fetch_add(1, std::memory_order_relaxed);
    Profiler* p = g_prof;
    t_open = false;
    if (!p || !p->on || !((p->mask >> tag) & 1ull)) return;
    if (p->pending.size() >= 16384) p->drain();
    t_begin = take_event(p);
    if (t_begin && cudaEventRecord(t_begin, s) == cudaSuccess) t_open = true;
}

void launch_end(int tag, cudaStream_t s) {
    Profiler* p = g_prof;
    if (g_rec || !p || !p->on) return;
    p->launches[tag] += 1;
    if (!((p->mask >> tag) & 1ull)) return;
    if (!t_open) return;
    t_open = false;
    cudaEvent_t e = take_event(p);
    if (!e) return;
    if (cudaEventRecord(e, s) != cudaSuccess) return;
    p->pending.push_back({t_begin, e, tag});
}

void Profiler::drain() {
    for (const Pending& q : pending) {
        float t = 0.f;
        if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess) ms[q.tag] += t;
        free_events.push_back(q.a);
        free_events.push_back(q.b);
    }
    pending.clear();
    cudaGetLastError();
}

Profiler::~Profiler() {
    drain();
    for (cudaEvent_t e : free_events) cudaEventDestroy(e);
}

long long total_launches() { return g_launches.load(); }

}  // namespace mfwq
