// Device-side BiCGStab (internal).
#pragma once

#include <cuda_runtime.h>

#include <functional>

#include "kernels.h"

namespace mfwq {

constexpr int kRedBlocks = 1024;  // largest reduction grid (deterministic sums)

// Blocks of the reductions of a solve of N unknowns: one per 2048 entries, at
// most kRedBlocks.  A fixed function of N, so a patch's sums are formed the
// same way in a separate and in a batched solve.
inline int red_blocks(size_t N) {
    const size_t b = (N + 2047) / 2048;
    return (int)(b < 1 ? 1 : (b > (size_t)kRedBlocks ? (size_t)kRedBlocks : b));
}

// Scalars of one BiCGStab solve, resident in device memory.
struct KScal {
    double rtol, tol2;
    double rho, rho_old, alpha, omega, beta;
    double s2, r2, f2;
    int skip1;   // solve finished: every kernel of the iteration returns at once
    int skip2;   // finished or converged on the half step: second half skipped
    int half, status, iters, pad;
};

template <typename T>
using LinOp = std::function<int(const T* in, T* out, const int* skip)>;

template <typename T>
struct KrylovBufs {
    T *r, *rhat, *p, *v, *s, *t, *ph, *sh;
};

// Solves A x = f with P as right preconditioner.  Synchronous.  *status is an
// MFWQ_* code (MFWQ_ENOCONV when maxit is reached); the return value reports
// launch failures only.
template <typename T>
int bicgstab(const LinOp<T>& A, const LinOp<T>& P, const T* f, T* x, bool x_given, double rtol, int maxit,
             const KrylovBufs<T>& b, KScal* dsc, KScal* hsc, double* part, size_t N, cudaStream_t s, int check_every,
             double* hist, int* iters, double* relres, int* status, int graph_chunk = 0);

// Enqueue-only pieces of the same solver (no host synchronisation), for
// callers that capture iterations into CUDA graphs: the init kernels, one
// iteration, and the conversion of a scalar block read back to the host.
template <typename T>
int krylov_enqueue_init(const LinOp<T>& A, const T* f, T* x, bool x_given, double rtol, const KrylovBufs<T>& b,
                        KScal* dsc, double* part, size_t N, cudaStream_t s);
template <typename T>
int krylov_enqueue_iter(const LinOp<T>& A, const LinOp<T>& P, const T* f, T* x, const KrylovBufs<T>& b, KScal* dsc,
                        double* part, size_t N, cudaStream_t s);
void krylov_result(const KScal& h, int* iters, double* relres, int* status);

template <typename T>
int axpby_into(const T* f, const T* v, T* r, size_t N, cudaStream_t s);  // r = f - v
int norm2_into(const double* x, size_t N, double* part, double* out, cudaStream_t s);  // *out = |x|^2
int to_f32_scaled(const double* x, const double* nrm2, float* y, size_t N, cudaStream_t s);   // y = x / |x|
int add_f32_scaled(double* u, const float* d, const double* nrm2, size_t N, cudaStream_t s);  // u += |x| d
template <typename S, typename D>
int convert_into(const S* x, D* y, size_t N, const int* skip, cudaStream_t s);  // y = x rounded to D (skip: no-op)

}  // namespace mfwq
