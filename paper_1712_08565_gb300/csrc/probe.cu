// Arithmetic-throughput probe (no counterpart in the paper): the measured
// denominator of the FP64- and FP32-pipe rooflines that the measurement
// reports beside the nominal unit counts.  Every thread runs 16 independent
// fused multiply-add chains in registers (the result is stored so the chains
// are not removed), at 4, 8 and 16 blocks of 256 threads per SM; the best
// rate counts.  Plain timing with CUDA events on the caller's stream; it
// changes no device setting.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "kernels.h"

namespace mfwq {
void set_last_error(const std::string& why);
}

namespace {

constexpr int kChains = 16;
constexpr int kIters = 8192;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(T* out, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int mfwq_probe_fma_rate(int fp64, void* stream, double* tflops) {
    if (!tflops) {
        mfwq::set_last_error("mfwq_probe_fma_rate: NULL output");
        return MFWQ_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        mfwq::set_last_error("mfwq_probe_fma_rate: no device");
        return MFWQ_ECUDA;
    }
    const size_t nmax = (size_t)sms * 16 * kProbeThreads;
    void* out = nullptr;
    if (cudaMalloc(&out, nmax * (fp64 ? sizeof(double) : sizeof(float))) != cudaSuccess) {
        cudaGetLastError();
        mfwq::set_last_error("mfwq_probe_fma_rate: device allocation failed");
        return MFWQ_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = MFWQ_OK;
    double best = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = MFWQ_ECUDA;
    for (int per_sm : {4, 8, 16}) {
        const int blocks = sms * per_sm;
        const double flops = 2.0 * (double)blocks * kProbeThreads * kChains * kIters;
        for (int rep = 0; rep < 4 && st == MFWQ_OK; ++rep) {  // the first launch warms up
            cudaEventRecord(e0, s);
            if (fp64) k_fma_probe<double><<<blocks, kProbeThreads, 0, s>>>((double*)out, 0.999999, 1e-7);
            else k_fma_probe<float><<<blocks, kProbeThreads, 0, s>>>((float*)out, 0.999999f, 1e-7f);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                st = MFWQ_ECUDA;
            else if (rep > 0 && ms > 0.f)
                best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (st != MFWQ_OK) {
        cudaGetLastError();
        mfwq::set_last_error("mfwq_probe_fma_rate: launch failed");
        return st;
    }
    *tflops = best;
    return MFWQ_OK;
}
