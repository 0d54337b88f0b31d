// Self-test of the bounded waits that guard every asynchronous copy and MMA
// completion in the library's kernels (no counterpart in the paper).
//
// The kernel arms an mbarrier for 16 bytes of transactions and issues no
// copy, so the phase can never complete: the wait must give up after its
// bound, record the timeout in the device error word and return, leaving the
// context usable.  Nothing is in flight when it returns, so nothing can land
// in the block's shared memory afterwards.
#include <cuda_runtime.h>

#include <string>

#include "kernels.h"
#include "ptx_async.cuh"

namespace mfwq {
void set_last_error(const std::string& why);
}

namespace {

__global__ void k_wait_selftest(long long limit, int* err) {
    __shared__ __align__(8) unsigned long long mbar;
    const uint32_t mb = mfwq::ptx::smem_u32(&mbar);
    if (threadIdx.x == 0) {
        mfwq::ptx::mbar_init(mb, 1);
        mfwq::ptx::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mfwq::ptx::mbar_expect_tx(mb, 16);  // 16 bytes that never arrive
    const bool ok = mfwq::ptx::mbar_wait(mb, 0, limit);
    if (!__syncthreads_and(ok ? 1 : 0) && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace

extern "C" int mfwq_selftest_bounded_wait(long long limit_cycles, void* stream) {
    if (limit_cycles < 1 || limit_cycles > mfwq::ptx::kWaitCycles) {
        mfwq::set_last_error("mfwq_selftest_bounded_wait: limit out of range");
        return MFWQ_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* derr = nullptr;
    if (cudaMalloc(&derr, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        mfwq::set_last_error("mfwq_selftest_bounded_wait: device allocation failed");
        return MFWQ_ENOMEM;
    }
    int st = MFWQ_OK, herr = 0;
    if (cudaMemsetAsync(derr, 0, sizeof(int), s) != cudaSuccess) st = MFWQ_ECUDA;
    if (st == MFWQ_OK) {
        k_wait_selftest<<<1, 64, 0, s>>>(limit_cycles, derr);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = MFWQ_ECUDA;
    }
    cudaFree(derr);
    if (st != MFWQ_OK) {
        mfwq::set_last_error("mfwq_selftest_bounded_wait: launch failed");
        return st;
    }
    if (herr) {
        mfwq::set_last_error("mfwq_selftest_bounded_wait: the wait gave up as designed");
        return MFWQ_ETIMEOUT;
    }
    mfwq::set_last_error("mfwq_selftest_bounded_wait: the wait completed although no copy was issued");
    return MFWQ_EINTERNAL;
}
