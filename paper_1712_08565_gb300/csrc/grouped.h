// Recording of kernel launches and their grouped execution over many patches
// (internal; used by the batched FP64 solve).
//
// While a Recorder is installed on the calling thread, the launchers of the
// operator, FD and Krylov kernels do not launch: each appends a LaunchRec (its
// kernel family and instance, its argument struct, the number of blocks it
// would launch and its device skip flag).  Recording one BiCGStab iteration
// per patch gives, for every patch, the same sequence of kernels that a
// separate solve launches, with that patch's arguments.  A grouped launch then
// runs stage k of all patches in one persistent kernel: its blocks walk a
// device table of (blocks, skip flag, arguments) per patch, skip the patches
// whose solve has finished, and call the same kernel bodies with a virtual
// block index, so each patch computes exactly what its own launch computes.
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <vector>

namespace mfwq {

// Kernel families and instances that can be grouped.
enum GroupKind {
    GK_NONE = 0,
    GK_VEC_P, GK_VEC_DOT_RV, GK_VEC_S, GK_VEC_DOT_TS, GK_VEC_XR,       // k_vec<double, OP>
    GK_FIN_DOT_RV, GK_FIN_S, GK_FIN_DOT_TS, GK_FIN_XR,                 // k_finish<OP>
    GK_FOLD, GK_UNFOLD,                                                // k_fold<UNFOLD>
    GK_DENSE_SLOW, GK_DENSE_FAST,                                      // k_dense_slow/fast<double>
    GK_SLOW_TRIAL_Z, GK_SLOW_TRIAL_Y, GK_SLOW_TEST_Y, GK_SLOW_TEST_Z,  // k_slow<Op<double>, 1>
    GK_XSTAGE0,                                                        // k_xstage_apply<double, 4, 0, 0>
    GK_OZ_SLICE, GK_OZ_PROD,                                           // k_oz_slice, k_fd_oz (split FP64 FD)
    GK_COUNT
};

struct LaunchRec {
    int kind = GK_NONE;
    int items = 0;                 // blocks of the patch's own launch
    int threads = 0, smem = 0;     // block size, dynamic shared memory
    const int* skip = nullptr;     // device flag: nonzero = the launch is a no-op
    std::vector<unsigned char> args;
};

struct Recorder {
    std::vector<LaunchRec> recs;
    bool unsupported = false;  // a launch that has no grouped form was requested
};

// Recorder of the calling thread (NULL: launches run normally).
extern thread_local Recorder* g_rec;

struct RecScope {
    Recorder* saved;
    explicit RecScope(Recorder* r) : saved(g_rec) { g_rec = r; }
    ~RecScope() { g_rec = saved; }
};

template <class A>
void record_launch(int kind, const A& a, int items, int threads, int smem, const int* skip) {
    LaunchRec r;
    r.kind = kind;
    r.items = items;
    r.threads = threads;
    r.smem = smem;
    r.skip = skip;
    r.args.resize(sizeof(A));
    std::memcpy(r.args.data(), &a, sizeof(A));
    g_rec->recs.push_back(std::move(r));
}

// Device table of one grouped stage: npatch slots of `stride` bytes, each
// {int items; int pad; const int* skip; argument struct at offset 16}.
constexpr int kSlotHeader = 16;

// Launches the grouped kernel of `kind` (owned by the file that defines the
// kernel family) over the table; false if the kind is not that file's.
bool grouped_launch_krylov(int kind, const unsigned char* tab, int stride, int npatch, int grid, int smem,
                           cudaStream_t s);
bool grouped_launch_fd(int kind, const unsigned char* tab, int stride, int npatch, int grid, int smem, cudaStream_t s);
bool grouped_launch_apply(int kind, const unsigned char* tab, int stride, int npatch, int grid, int smem, cudaStream_t s);
bool grouped_launch_xstage(int kind, const unsigned char* tab, int stride, int npatch, int grid, int smem,
                           cudaStream_t s);
bool grouped_launch_oz(int kind, const unsigned char* tab, int stride, int npatch, int grid, int smem, cudaStream_t s);
// Raises the dynamic shared-memory limit of the grouped kernels that take it.
int configure_grouped_smem(int bytes);

#ifdef __CUDACC__
constexpr int kGroupMax = 1024;   // patches of one grouped launch (shared-memory slot headers)
constexpr int kGroupArgs = 1024;  // bytes of one patch's argument struct held in shared memory

// Runs f(args, item) for every item of every patch whose skip flag is clear,
// items spread over the grid (patch p's items start at a rotated block so
// that consecutive patches start on different blocks).  The slot headers
// (item count, skip flag) are read once per block, and a patch's argument
// struct is copied into shared memory before its items run, so the bodies
// read their arguments from shared memory rather than global memory.  With
// SYNC a barrier follows every item (bodies that reuse shared memory).
template <class A, bool SYNC, class F>
__device__ __forceinline__ void grouped_for(const unsigned char* __restrict__ tab, int stride, int npatch, F&& f) {
    static_assert(sizeof(A) <= kGroupArgs, "argument struct too large for the grouped launch");
    __shared__ int s_items[kGroupMax];
    __shared__ unsigned char s_live[kGroupMax];
    __shared__ __align__(16) unsigned char s_args[kGroupArgs];
    for (int p = threadIdx.x; p < npatch; p += blockDim.x) {
        const unsigned char* slot = tab + (size_t)p * stride;
        const int* skip = *reinterpret_cast<const int* const*>(slot + 8);
        s_items[p] = *reinterpret_cast<const int*>(slot);
        s_live[p] = (skip && *skip) ? 0 : 1;
    }
    __syncthreads();
    int base = 0;
    for (int p = 0; p < npatch; ++p) {
        const int n = s_items[p];
        int first = (int)blockIdx.x - (int)(base % (int)gridDim.x);
        if (first < 0) first += gridDim.x;
        base += n;
        if (!s_live[p] || first >= n) continue;
        const int4* src = reinterpret_cast<const int4*>(tab + (size_t)p * stride + kSlotHeader);
        for (int w = threadIdx.x; w < (int)((sizeof(A) + 15) / 16); w += blockDim.x)
            reinterpret_cast<int4*>(s_args)[w] = src[w];
        __syncthreads();
        const A& a = *reinterpret_cast<const A*>(s_args);
        for (int it = first; it < n; it += gridDim.x) {
            f(a, it);
            if (SYNC) __syncthreads();
        }
        __syncthreads();  // s_args is rewritten for the next patch
    }
}
#endif

}  // namespace mfwq
