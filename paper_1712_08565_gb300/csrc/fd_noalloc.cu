// FD preconditioner entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// preconditioner: code that runs while a CUDA graph is being captured in
// global mode (allocation is illegal then), code whose process has handed
// all device memory to a framework's caching allocator, or code with a fixed
// memory budget that must not allocate per call.  mfwq_fd_precond_noalloc
// serves them: the caller passes the inputs (the FD factors and r) and the
// output z, and the one intermediate tensor the six mode products need lives
// in a fixed array of device memory that is part of the library's module.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.h"

namespace mfwq {
void set_last_error(const std::string& why);
}

namespace {

constexpr size_t kNoAllocMaxN = MFWQ_NOALLOC_MAX_N;  // doubles: 32 MB
constexpr int kMaxDevices = 64;

// Scratch of every call on this device.  It belongs to the module, so every
// GPU that loads the library holds these 32 MB until the process exits.
static __device__ __align__(256) double g_fd_scratch[kNoAllocMaxN];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_fd_scratch on the current device, looked up once per
// device (host code cannot use the symbol itself as a device address).
int scratch_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        mfwq::set_last_error("mfwq_fd_precond_noalloc: no usable current device");
        return MFWQ_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fd_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            mfwq::set_last_error(std::string("mfwq_fd_precond_noalloc: cudaGetSymbolAddress failed: ") +
                                 cudaGetErrorString(e));
            return MFWQ_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return MFWQ_OK;
}

// True if p is device (or managed) memory that device dev can address as its
// own: allocated on dev, or managed.  Host memory, pinned host memory and
// other devices' memory are refused.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int mfwq_fd_precond_noalloc(const int n[3], const double* const U_dev[3], const double* const UT_dev[3],
                                       const double* const lam_dev[3], const double* r_dev, double* z_dev, void* stream) {
    if (!n || !U_dev || !UT_dev || !lam_dev || !r_dev || !z_dev || r_dev == z_dev) {
        mfwq::set_last_error("mfwq_fd_precond_noalloc: NULL or aliased argument");
        return MFWQ_EINVAL;
    }
    size_t N = 1;
    for (int l = 0; l < 3; ++l) {
        if (n[l] < 1 || !U_dev[l] || !UT_dev[l] || !lam_dev[l]) {
            mfwq::set_last_error("mfwq_fd_precond_noalloc: bad size or factor pointer in direction " + std::to_string(l + 1));
            return MFWQ_EINVAL;
        }
        // reject before multiplying, so that no product can wrap around
        if ((size_t)n[l] > kNoAllocMaxN / N) {
            mfwq::set_last_error("mfwq_fd_precond_noalloc: n1*n2*n3 exceeds the fixed scratch of " +
                                 std::to_string(kNoAllocMaxN) + " doubles");
            return MFWQ_EINVAL;
        }
        N *= (size_t)n[l];
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        mfwq::set_last_error("mfwq_fd_precond_noalloc: no usable current device");
        return MFWQ_ECUDA;
    }
    // every buffer must be device memory of the current device: the scratch
    // address below is this device's, and a kernel given another device's (or
    // host) memory would fault or read the wrong memory
    for (int l = 0; l < 3; ++l) {
        if (!on_device(U_dev[l], dev) || !on_device(UT_dev[l], dev) || !on_device(lam_dev[l], dev)) {
            mfwq::set_last_error("mfwq_fd_precond_noalloc: an FD factor of direction " + std::to_string(l + 1) +
                                 " is not device memory of the current device " + std::to_string(dev));
            return MFWQ_EINVAL;
        }
    }
    if (!on_device(r_dev, dev) || !on_device(z_dev, dev)) {
        mfwq::set_last_error("mfwq_fd_precond_noalloc: r or z is not device memory of the current device " +
                             std::to_string(dev));
        return MFWQ_EINVAL;
    }
    double* scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st != MFWQ_OK) return st;
    mfwq::DirD<double> d[3] = {};
    for (int l = 0; l < 3; ++l) {
        d[l].n = n[l];
        d[l].U = U_dev[l];
        d[l].UT = UT_dev[l];
        d[l].lam = lam_dev[l];
    }
    // Every pass writes its whole output before the next one reads it, so the
    // scratch needs no clearing between calls.
    st = mfwq::run_fd64(d, r_dev, z_dev, scratch, nullptr, static_cast<cudaStream_t>(stream));
    if (st != MFWQ_OK) mfwq::set_last_error("mfwq_fd_precond_noalloc: kernel launch failed");
    return st;
}
