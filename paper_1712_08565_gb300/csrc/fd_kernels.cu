// Fast Diagonalization preconditioner (Section 4; Lynch et al.'s method in
// the form used by Sangalli & Tani): with U_l^T M_l U_l = I and
// U_l^T K_l U_l = diag(lambda_l),
//   P^-1 r = (U3 (x) U2 (x) U1) diag(1 / (l1_i + l2_j + l3_k)) (U3 (x) U2 (x) U1)^T r,
// i.e. three dense mode products with U_l^T, a pointwise scaling, and three
// with U_l.  This file holds the SIMT versions (FP64 on the FP64 pipe, and an
// FP32 one); the tensor-core TF32/BF16 version is in fd_tc.cu.
#include <cuda_runtime.h>

#include "kernels.h"
#include "prof.h"

namespace mfwq {
namespace {

constexpr int kThreads = 256;
constexpr int kRT = 4;  // output rows per thread (slow dims)
constexpr int kAT = 4;  // output rows per thread (fast dim)

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// out[a][r][c] = sum_t M[r][t] in[a][t][c], r, t < n (dims 2 and 3).  With
// scale != NULL (forward pass along dim 3, A = 1): out /= l3[r] + l2[j] + l1[i],
// c = j n1 + i.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dense_slow(const T* __restrict__ M, const T* __restrict__ in, T* __restrict__ out,
                                                         int A, int n, int C, const T* __restrict__ l1,
                                                         const T* __restrict__ l2, const T* __restrict__ l3, int n1,
                                                         const int* skip) {
    if (skip && *skip) return;
    const int r0 = blockIdx.y * kRT;
    const int nr = min(kRT, n - r0);
    const size_t AC = (size_t)A * C;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < AC; e += (size_t)gridDim.x * blockDim.x) {
        const size_t a = e / C, c = e - a * C;
        const T* x = in + a * (size_t)n * C + c;
        T acc[kRT];
#pragma unroll
        for (int k = 0; k < kRT; ++k) acc[k] = 0;
        if (nr == kRT) {
            for (int t = 0; t < n; ++t) {
                const T v = x[(size_t)t * C];
#pragma unroll
                for (int k = 0; k < kRT; ++k) acc[k] = fmaT(M[(size_t)(r0 + k) * n + t], v, acc[k]);
            }
        } else {
            for (int t = 0; t < n; ++t) {
                const T v = x[(size_t)t * C];
                for (int k = 0; k < nr; ++k) acc[k] = fmaT(M[(size_t)(r0 + k) * n + t], v, acc[k]);
            }
        }
        for (int k = 0; k < nr; ++k) {
            T val = acc[k];
            if (l3) {
                const int j = (int)(c / n1), i = (int)(c - (size_t)j * n1);
                val = val / (l3[r0 + k] + l2[j] + l1[i]);
            }
            out[(a * n + r0 + k) * (size_t)C + c] = val;
        }
    }
}

// out[a][r] = sum_t M[r][t] in[a][t] (dim 1), MT[t][r] = M[r][t].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dense_fast(const T* __restrict__ MT, const T* __restrict__ in, T* __restrict__ out,
                                                         int A, int n, const int* skip) {
    if (skip && *skip) return;
    const int groups = (A + kAT - 1) / kAT;
    const size_t total = (size_t)groups * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(e / n), r = (int)(e - (size_t)g * n);
        const int a0 = g * kAT;
        const int na = min(kAT, A - a0);
        T acc[kAT];
#pragma unroll
        for (int k = 0; k < kAT; ++k) acc[k] = 0;
        const T* x = in + (size_t)a0 * n;
        if (na == kAT) {
            for (int t = 0; t < n; ++t) {
                const T m = MT[(size_t)t * n + r];
#pragma unroll
                for (int k = 0; k < kAT; ++k) acc[k] = fmaT(m, x[(size_t)k * n + t], acc[k]);
            }
        } else {
            for (int t = 0; t < n; ++t) {
                const T m = MT[(size_t)t * n + r];
                for (int k = 0; k < na; ++k) acc[k] = fmaT(m, x[(size_t)k * n + t], acc[k]);
            }
        }
        for (int k = 0; k < na; ++k) out[(size_t)(a0 + k) * n + r] = acc[k];
    }
}

template <typename T>
cudaError_t dense_slow(const T* M, const T* in, T* out, int A, int n, int C, const T* l1, const T* l2, const T* l3, int n1,
                       const int* skip, cudaStream_t s) {
    size_t AC = (size_t)A * C;
    unsigned bx = (unsigned)((AC + kThreads - 1) / kThreads);
    if (bx > 65535u) bx = 65535u;
    dim3 grid(bx, (n + kRT - 1) / kRT);
    launch_begin(S_FD_DIM23, s);
    k_dense_slow<T><<<grid, kThreads, 0, s>>>(M, in, out, A, n, C, l1, l2, l3, n1, skip);
    launch_end(S_FD_DIM23, s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dense_fast(const T* MT, const T* in, T* out, int A, int n, const int* skip, cudaStream_t s) {
    size_t total = (size_t)((A + kAT - 1) / kAT) * n;
    size_t blocks = (total + kThreads - 1) / kThreads;
    if (blocks > 1u << 20) blocks = 1u << 20;
    launch_begin(S_FD_DIM1, s);
    k_dense_fast<T><<<(unsigned)blocks, kThreads, 0, s>>>(MT, in, out, A, n, skip);
    launch_end(S_FD_DIM1, s);
    return cudaGetLastError();
}

// Forward (U^T) and backward (U) transforms of the FD apply.
template <typename T>
int run_fd_simt(const DirD<T> d[3], const T* r, T* z, T* tmp, const int* skip, cudaStream_t s) {
    const int n1 = d[0].n, n2 = d[1].n, n3 = d[2].n;
    // dim 1 with U1^T: M = U1^T, MT = U1
    if (dense_fast<T>(d[0].U, r, tmp, n3 * n2, n1, skip, s) != cudaSuccess) return MFWQ_ECUDA;
    // dim 2 with U2^T
    if (dense_slow<T>(d[1].UT, tmp, z, n3, n2, n1, nullptr, nullptr, nullptr, n1, skip, s) != cudaSuccess) return MFWQ_ECUDA;
    // dim 3 with U3^T, then divide by l1 + l2 + l3
    if (dense_slow<T>(d[2].UT, z, tmp, 1, n3, n2 * n1, d[0].lam, d[1].lam, d[2].lam, n1, skip, s) != cudaSuccess)
        return MFWQ_ECUDA;
    // backward: dim 3 with U3, dim 2 with U2, dim 1 with U1 (MT = U1^T)
    if (dense_slow<T>(d[2].U, tmp, z, 1, n3, n2 * n1, nullptr, nullptr, nullptr, n1, skip, s) != cudaSuccess) return MFWQ_ECUDA;
    if (dense_slow<T>(d[1].U, z, tmp, n3, n2, n1, nullptr, nullptr, nullptr, n1, skip, s) != cudaSuccess) return MFWQ_ECUDA;
    if (dense_fast<T>(d[0].UT, tmp, z, n3 * n2, n1, skip, s) != cudaSuccess) return MFWQ_ECUDA;
    return MFWQ_OK;
}

}  // namespace

int run_fd64(const DirD<double> d[3], const double* r, double* z, double* tmp, const int* skip, cudaStream_t s) {
    return run_fd_simt<double>(d, r, z, tmp, skip, s);
}

int run_fd32_simt(const DirD<float> d[3], const float* r, float* z, float* tmp, const int* skip, cudaStream_t s) {
    return run_fd_simt<float>(d, r, z, tmp, skip, s);
}

}  // namespace mfwq
