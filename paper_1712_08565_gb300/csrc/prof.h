// Per-stage launch counting and optional CUDA-event timing (internal).
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace mfwq {

// Stage tags, in the order of mfwq_stage_name().
enum StageTag {
    S_TRIAL_Z = 0, S_TRIAL_Y, S_XSTAGE, S_TEST_Y, S_TEST_Z,
    S_TEST_ZT, S_TEST_YT, S_XSTAGE_T, S_TRIAL_YT, S_TRIAL_ZT, S_XSTAGE_GRAD,
    S_FD_DIM1, S_FD_DIM23, S_FD_TC, S_KRYLOV, S_SETUP, S_FD_FOLD, S_MASS, S_H1, S_FUSED, S_FD_OZ, S_NTAGS
};

struct Profiler {
    bool on = false;
    unsigned long long mask = ~0ull;  // stages bracketed by events while on (bit = stage tag)
    struct Pending {
        cudaEvent_t a, b;
        int tag;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    double ms[S_NTAGS] = {};
    long long launches[S_NTAGS] = {};
    ~Profiler();
    void drain();
};

// Profiler of the C-ABI call running on this thread (NULL: none).
extern thread_local Profiler* g_prof;

struct ProfScope {
    Profiler* saved;
    explicit ProfScope(Profiler* p) : saved(g_prof) { g_prof = p; }
    ~ProfScope() { g_prof = saved; }
};

// Bracket every kernel launch: counts it and, when the current profiler is
// on, records a CUDA event before and after it on the launch stream.
void launch_begin(int tag, cudaStream_t s);
void launch_end(int tag, cudaStream_t s);

// Kernels launched by this library in this process so far.
long long total_launches();

}  // namespace mfwq
