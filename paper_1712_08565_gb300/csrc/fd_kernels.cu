// Fast Diagonalization preconditioner (Section 4; Lynch et al.'s method in
// the form used by Sangalli & Tani): with U_l^T M_l U_l = I and
// U_l^T K_l U_l = diag(lambda_l),
//   P^-1 r = (U3 (x) U2 (x) U1) diag(1 / (l1_i + l2_j + l3_k)) (U3 (x) U2 (x) U1)^T r,
// i.e. three dense mode products with U_l^T, a pointwise scaling, and three
// with U_l.  This file holds the SIMT versions (FP64 on the FP64 pipe, and an
// FP32 one); the tensor-core TF32/BF16 version is in fd_tc.cu.
#include <cuda_runtime.h>

#include "grouped.h"
#include "kernels.h"
#include "prof.h"

namespace mfwq {
namespace {

constexpr int kThreads = 256;
constexpr int kRT = 4;  // output rows per thread (slow dims)
constexpr int kAT = 4;  // output rows per thread (fast dim)
// Threads per block of the two dense mode-product launches: finer than 256, so
// the last blocks of a launch leave less of the FP64 pipe idle (FD at 130^3:
// 1.72 -> 1.61 ms).
constexpr int kDenseThreads = 128;

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// Mode product along a middle or slowest dimension of extent ld:
// out[a][outoff + r][c] = sum_{t < nin} M[r][t] in[a][inoff + t][c], r < nout
// (M row-major nout x nin).  With l3 != NULL (forward pass along dimension 3,
// A = 1): out /= l3[outoff + r] + l2[j] + l1[i], c = j n1 + i.
template <typename T>
struct DenseSlowArgs {
    const T* M;
    const T* in;
    T* out;
    int A, ld, nin, nout, inoff, outoff, C;
    const T* l1;
    const T* l2;
    const T* l3;
    int n1;
    int gx;  // blocks along the columns
};

// One block (bx, by) of gx column blocks.
template <typename T>
__device__ __forceinline__ void dense_slow_body(const DenseSlowArgs<T>& p, int bx, int by) {
    const T* __restrict__ M = p.M;
    const T* __restrict__ in = p.in;
    T* __restrict__ out = p.out;
    const int A = p.A, ld = p.ld, nin = p.nin, nout = p.nout, inoff = p.inoff, outoff = p.outoff, C = p.C, n1 = p.n1;
    const T* __restrict__ l1 = p.l1;
    const T* __restrict__ l2 = p.l2;
    const T* __restrict__ l3 = p.l3;
    const int r0 = by * kRT;
    const int nr = min(kRT, nout - r0);
    const size_t AC = (size_t)A * C;
    for (size_t e = (size_t)bx * blockDim.x + threadIdx.x; e < AC; e += (size_t)p.gx * blockDim.x) {
        const size_t a = e / C, c = e - a * C;
        const T* x = in + (a * ld + inoff) * (size_t)C + c;
        T acc[kRT];
#pragma unroll
        for (int k = 0; k < kRT; ++k) acc[k] = 0;
        if (nr == kRT) {
            for (int t = 0; t < nin; ++t) {
                const T v = x[(size_t)t * C];
#pragma unroll
                for (int k = 0; k < kRT; ++k) acc[k] = fmaT(M[(size_t)(r0 + k) * nin + t], v, acc[k]);
            }
        } else {
            for (int t = 0; t < nin; ++t) {
                const T v = x[(size_t)t * C];
                for (int k = 0; k < nr; ++k) acc[k] = fmaT(M[(size_t)(r0 + k) * nin + t], v, acc[k]);
            }
        }
        for (int k = 0; k < nr; ++k) {
            T val = acc[k];
            if (l3) {
                const int j = (int)(c / n1), i = (int)(c - (size_t)j * n1);
                val = val / (l3[outoff + r0 + k] + l2[j] + l1[i]);
            }
            out[(a * ld + outoff + r0 + k) * (size_t)C + c] = val;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_dense_slow(DenseSlowArgs<T> p, const int* skip) {
    if (skip && *skip) return;
    dense_slow_body<T>(p, blockIdx.x, blockIdx.y);
}

// Mode product along the fastest dimension of extent ld:
// out[a][outoff + r] = sum_{t < nin} MT[t][r] in[a][inoff + t], r < nout
// (MT row-major nin x nout, i.e. M transposed, so lanes read it coalesced).
template <typename T>
struct DenseFastArgs {
    const T* MT;
    const T* in;
    T* out;
    int A, ld, nin, nout, inoff, outoff;
    int gx;  // blocks
};

template <typename T>
__device__ __forceinline__ void dense_fast_body(const DenseFastArgs<T>& p, int bx) {
    const T* __restrict__ MT = p.MT;
    const T* __restrict__ in = p.in;
    T* __restrict__ out = p.out;
    const int A = p.A, ld = p.ld, nin = p.nin, nout = p.nout, inoff = p.inoff, outoff = p.outoff;
    const int groups = (A + kAT - 1) / kAT;
    const size_t total = (size_t)groups * nout;
    for (size_t e = (size_t)bx * blockDim.x + threadIdx.x; e < total; e += (size_t)p.gx * blockDim.x) {
        const int g = (int)(e / nout), r = (int)(e - (size_t)g * nout);
        const int a0 = g * kAT;
        const int na = min(kAT, A - a0);
        T acc[kAT];
#pragma unroll
        for (int k = 0; k < kAT; ++k) acc[k] = 0;
        const T* x = in + (size_t)a0 * ld + inoff;
        if (na == kAT) {
            for (int t = 0; t < nin; ++t) {
                const T m = MT[(size_t)t * nout + r];
#pragma unroll
                for (int k = 0; k < kAT; ++k) acc[k] = fmaT(m, x[(size_t)k * ld + t], acc[k]);
            }
        } else {
            for (int t = 0; t < nin; ++t) {
                const T m = MT[(size_t)t * nout + r];
                for (int k = 0; k < na; ++k) acc[k] = fmaT(m, x[(size_t)k * ld + t], acc[k]);
            }
        }
        for (int k = 0; k < na; ++k) out[(size_t)(a0 + k) * ld + outoff + r] = acc[k];
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_dense_fast(DenseFastArgs<T> p, const int* skip) {
    if (skip && *skip) return;
    dense_fast_body<T>(p, blockIdx.x);
}

// Even/odd folding along a dimension of extent n (h = n/2, he = n - h):
// out[j] = in[j] + in[n-1-j] (j < h), out[h] = in[h] (odd n),
// out[he + j] = in[j] - in[n-1-j] (j < h); and its inverse-type unfold
// out[j] = in[j] + in[he+j], out[n-1-j] = in[j] - in[he+j], out[h] = in[h].
struct FoldArgs {
    const double* in;
    double* out;
    int A, n, C;
    int gx;  // blocks
};

template <bool UNFOLD>
__device__ __forceinline__ void fold_body(const FoldArgs& p, int bx) {
    const double* __restrict__ in = p.in;
    double* __restrict__ out = p.out;
    const int A = p.A, n = p.n, C = p.C;
    const int h = n / 2, he = n - h;
    const size_t total = (size_t)A * n * C;
    for (size_t e = (size_t)bx * blockDim.x + threadIdx.x; e < total; e += (size_t)p.gx * blockDim.x) {
        const size_t c = e % C;
        const size_t aj = e / C;
        const int j = (int)(aj % n);
        const size_t base = (aj - j) * C + c;  // element (a, 0, c)
        double v;
        if (!UNFOLD) {
            if (j < h) v = in[base + (size_t)j * C] + in[base + (size_t)(n - 1 - j) * C];
            else if (j < he) v = in[base + (size_t)j * C];
            else v = in[base + (size_t)(j - he) * C] - in[base + (size_t)(n - 1 - (j - he)) * C];
        } else {
            if (j < h) v = in[base + (size_t)j * C] + in[base + (size_t)(he + j) * C];
            else if (j < he) v = in[base + (size_t)j * C];
            else {
                const int jj = n - 1 - j;
                v = in[base + (size_t)jj * C] - in[base + (size_t)(he + jj) * C];
            }
        }
        out[e] = v;
    }
}

template <bool UNFOLD>
__global__ void __launch_bounds__(kThreads) k_fold(FoldArgs p, const int* skip) {
    if (skip && *skip) return;
    fold_body<UNFOLD>(p, blockIdx.x);
}

// ---- grouped forms (batched FP64 solve)
__global__ void __launch_bounds__(kThreads) k_dense_slow_grouped(const unsigned char* __restrict__ tab, int stride,
                                                                 int npatch) {
    grouped_for<DenseSlowArgs<double>, false>(tab, stride, npatch, [&](const DenseSlowArgs<double>& p, int item) {
        const int by = item / p.gx;
        dense_slow_body<double>(p, item - by * p.gx, by);
    });
}
__global__ void __launch_bounds__(kThreads) k_dense_fast_grouped(const unsigned char* __restrict__ tab, int stride,
                                                                 int npatch) {
    grouped_for<DenseFastArgs<double>, false>(tab, stride, npatch,
                                       [&](const DenseFastArgs<double>& p, int item) { dense_fast_body<double>(p, item); });
}
template <bool UNFOLD>
__global__ void __launch_bounds__(kThreads) k_fold_grouped(const unsigned char* __restrict__ tab, int stride, int npatch) {
    grouped_for<FoldArgs, false>(tab, stride, npatch, [&](const FoldArgs& p, int item) { fold_body<UNFOLD>(p, item); });
}

template <typename T>
cudaError_t dense_slow(const T* M, const T* in, T* out, int A, int ld, int nin, int nout, int inoff, int outoff, int C,
                       const T* l1, const T* l2, const T* l3, int n1, const int* skip, cudaStream_t s) {
    size_t AC = (size_t)A * C;
    unsigned bx = (unsigned)((AC + kDenseThreads - 1) / kDenseThreads);
    if (bx > 65535u) bx = 65535u;
    dim3 grid(bx, (nout + kRT - 1) / kRT);
    DenseSlowArgs<T> p{M, in, out, A, ld, nin, nout, inoff, outoff, C, l1, l2, l3, n1, (int)bx};
    if (g_rec) {
        if (sizeof(T) != 8) g_rec->unsupported = true;
        else record_launch(GK_DENSE_SLOW, p, (int)(grid.x * grid.y), kDenseThreads, 0, skip);
        return cudaSuccess;
    }
    launch_begin(S_FD_DIM23, s);
    k_dense_slow<T><<<grid, kDenseThreads, 0, s>>>(p, skip);
    launch_end(S_FD_DIM23, s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dense_fast(const T* MT, const T* in, T* out, int A, int ld, int nin, int nout, int inoff, int outoff,
                       const int* skip, cudaStream_t s) {
    size_t total = (size_t)((A + kAT - 1) / kAT) * nout;
    size_t blocks = (total + kDenseThreads - 1) / kDenseThreads;
    if (blocks > 1u << 20) blocks = 1u << 20;
    DenseFastArgs<T> p{MT, in, out, A, ld, nin, nout, inoff, outoff, (int)blocks};
    if (g_rec) {
        if (sizeof(T) != 8) g_rec->unsupported = true;
        else record_launch(GK_DENSE_FAST, p, (int)blocks, kDenseThreads, 0, skip);
        return cudaSuccess;
    }
    launch_begin(S_FD_DIM1, s);
    k_dense_fast<T><<<(unsigned)blocks, kDenseThreads, 0, s>>>(p, skip);
    launch_end(S_FD_DIM1, s);
    return cudaGetLastError();
}

template <bool UNFOLD>
cudaError_t fold(const double* in, double* out, int A, int n, int C, const int* skip, cudaStream_t s) {
    size_t total = (size_t)A * n * C;
    size_t blocks = (total + kThreads - 1) / kThreads;
    if (blocks > 1u << 20) blocks = 1u << 20;
    FoldArgs p{in, out, A, n, C, (int)blocks};
    if (g_rec) {
        record_launch(UNFOLD ? GK_UNFOLD : GK_FOLD, p, (int)blocks, kThreads, 0, skip);
        return cudaSuccess;
    }
    launch_begin(S_FD_FOLD, s);
    k_fold<UNFOLD><<<(unsigned)blocks, kThreads, 0, s>>>(p, skip);
    launch_end(S_FD_FOLD, s);
    return cudaGetLastError();
}

// Forward (U^T) and backward (U) transforms of the FD apply.
template <typename T>
int run_fd_simt(const DirD<T> d[3], const T* r, T* z, T* tmp, const int* skip, cudaStream_t s) {
    const int n1 = d[0].n, n2 = d[1].n, n3 = d[2].n;
    // dim 1 with U1^T: M = U1^T, MT = U1
    if (dense_fast<T>(d[0].U, r, tmp, n3 * n2, n1, n1, n1, 0, 0, skip, s) != cudaSuccess) return MFWQ_ECUDA;
    // dim 2 with U2^T
    if (dense_slow<T>(d[1].UT, tmp, z, n3, n2, n2, n2, 0, 0, n1, nullptr, nullptr, nullptr, n1, skip, s) != cudaSuccess)
        return MFWQ_ECUDA;
    // dim 3 with U3^T, then divide by l1 + l2 + l3
    if (dense_slow<T>(d[2].UT, z, tmp, 1, n3, n3, n3, 0, 0, n2 * n1, d[0].lam, d[1].lam, d[2].lam, n1, skip, s) != cudaSuccess)
        return MFWQ_ECUDA;
    // backward: dim 3 with U3, dim 2 with U2, dim 1 with U1 (MT = U1^T)
    if (dense_slow<T>(d[2].U, tmp, z, 1, n3, n3, n3, 0, 0, n2 * n1, nullptr, nullptr, nullptr, n1, skip, s) != cudaSuccess)
        return MFWQ_ECUDA;
    if (dense_slow<T>(d[1].U, z, tmp, n3, n2, n2, n2, 0, 0, n1, nullptr, nullptr, nullptr, n1, skip, s) != cudaSuccess)
        return MFWQ_ECUDA;
    if (dense_fast<T>(d[0].UT, tmp, z, n3 * n2, n1, n1, n1, 0, 0, skip, s) != cudaSuccess) return MFWQ_ECUDA;
    return MFWQ_OK;
}

// Same transforms with the even/odd split of every direction (knot vectors
// symmetric about 1/2): each mode product becomes a fold pass and two
// half-size products, halving the FP64 work.  Buffers alternate between tmp
// and z; r is not written.
int run_fd_split(const DirD<double> d[3], const double* r, double* z, double* tmp, const int* skip, cudaStream_t s) {
    const int n1 = d[0].n, n2 = d[1].n, n3 = d[2].n;
    double* T1 = tmp;
    double* T2 = z;
#define FD_TRY(x)                                 \
    do {                                          \
        if ((x) != cudaSuccess) return MFWQ_ECUDA; \
    } while (0)
    // ---- forward
    // dim 1: fold rows, even and odd products (MT = V, row-major)
    FD_TRY(fold<false>(r, T1, n3 * n2, n1, 1, skip, s));
    FD_TRY(dense_fast<double>(d[0].Ve, T1, T2, n3 * n2, n1, d[0].he, d[0].he, 0, 0, skip, s));
    FD_TRY(dense_fast<double>(d[0].Vo, T1, T2, n3 * n2, n1, d[0].ho, d[0].ho, d[0].he, d[0].he, skip, s));
    // dim 2 (M = V^T)
    FD_TRY(fold<false>(T2, T1, n3, n2, n1, skip, s));
    FD_TRY(dense_slow<double>(d[1].VeT, T1, T2, n3, n2, d[1].he, d[1].he, 0, 0, n1, nullptr, nullptr, nullptr, n1, skip, s));
    FD_TRY(dense_slow<double>(d[1].VoT, T1, T2, n3, n2, d[1].ho, d[1].ho, d[1].he, d[1].he, n1, nullptr, nullptr, nullptr,
                              n1, skip, s));
    // dim 3 and the Kronecker-sum scaling (eigenvalues in split order in every direction)
    FD_TRY(fold<false>(T2, T1, 1, n3, n2 * n1, skip, s));
    FD_TRY(dense_slow<double>(d[2].VeT, T1, T2, 1, n3, d[2].he, d[2].he, 0, 0, n2 * n1, d[0].lam_split, d[1].lam_split,
                              d[2].lam_split, n1, skip, s));
    FD_TRY(dense_slow<double>(d[2].VoT, T1, T2, 1, n3, d[2].ho, d[2].ho, d[2].he, d[2].he, n2 * n1, d[0].lam_split,
                              d[1].lam_split, d[2].lam_split, n1, skip, s));
    // ---- backward: products with V (M = V), then unfold
    FD_TRY(dense_slow<double>(d[2].Ve, T2, T1, 1, n3, d[2].he, d[2].he, 0, 0, n2 * n1, nullptr, nullptr, nullptr, n1, skip, s));
    FD_TRY(dense_slow<double>(d[2].Vo, T2, T1, 1, n3, d[2].ho, d[2].ho, d[2].he, d[2].he, n2 * n1, nullptr, nullptr, nullptr,
                              n1, skip, s));
    FD_TRY(fold<true>(T1, T2, 1, n3, n2 * n1, skip, s));
    FD_TRY(dense_slow<double>(d[1].Ve, T2, T1, n3, n2, d[1].he, d[1].he, 0, 0, n1, nullptr, nullptr, nullptr, n1, skip, s));
    FD_TRY(dense_slow<double>(d[1].Vo, T2, T1, n3, n2, d[1].ho, d[1].ho, d[1].he, d[1].he, n1, nullptr, nullptr, nullptr, n1,
                              skip, s));
    FD_TRY(fold<true>(T1, T2, n3, n2, n1, skip, s));
    FD_TRY(dense_fast<double>(d[0].VeT, T2, T1, n3 * n2, n1, d[0].he, d[0].he, 0, 0, skip, s));
    FD_TRY(dense_fast<double>(d[0].VoT, T2, T1, n3 * n2, n1, d[0].ho, d[0].ho, d[0].he, d[0].he, skip, s));
    FD_TRY(fold<true>(T1, z, n3 * n2, n1, 1, skip, s));
#undef FD_TRY
    return MFWQ_OK;
}

}  // namespace

bool grouped_launch_fd(int kind, const unsigned char* tab, int stride, int npatch, int grid, int smem, cudaStream_t s) {
    (void)smem;
    switch (kind) {
        case GK_DENSE_SLOW: k_dense_slow_grouped<<<grid, kDenseThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_DENSE_FAST: k_dense_fast_grouped<<<grid, kDenseThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_FOLD: k_fold_grouped<false><<<grid, kThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_UNFOLD: k_fold_grouped<true><<<grid, kThreads, 0, s>>>(tab, stride, npatch); return true;
        default: return false;
    }
}

int run_fd64(const DirD<double> d[3], const double* r, double* z, double* tmp, const int* skip, cudaStream_t s) {
    if (d[0].sym && d[1].sym && d[2].sym) return run_fd_split(d, r, z, tmp, skip, s);
    return run_fd_simt<double>(d, r, z, tmp, skip, s);
}

int run_fd32_simt(const DirD<float> d[3], const float* r, float* z, float* tmp, const int* skip, cudaStream_t s) {
    return run_fd_simt<float>(d, r, z, tmp, skip, s);
}

}  // namespace mfwq
