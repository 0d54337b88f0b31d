// Kernel launchers shared by the C-ABI layer (internal).
#pragma once

#include <cuda_runtime.h>

#include "mfwq_internal.h"

namespace mfwq {

// Everything one operator application needs, in one precision.
template <typename T>
struct OpCtx {
    DirD<T> d[3];
    const T* C;        // [6][cs]: field s at C + s * cs, Nq values each
    size_t Nq;         // quadrature points
    size_t cs;         // field stride of C, a multiple of 32
    T* scratch;        // apply_scratch_elems() elements of T
    cudaStream_t stream;
    int xlines = 4;    // (q3, q2) lines per block of the forward x stage: 2, 4 or 8
    int xmode = 0;     // forward x-stage work mapping: 0 per (line, item), 1 per item over all lines,
                       // 2 and 3 the same with the block's inputs prefetched by bulk copies,
                       // 4 and 5 two-row tiles over 4 or 8 lines (8 lines per block)
    int xcarve = 0;    // 1: forward x stage with the reduced shared-memory carveout (larger L1)
    int srows = 1;     // output rows per thread of the slow-dimension stages: 1, 2 or 4
    int* err = nullptr;  // device error word: set when a bounded wait times out
    const T* cm = nullptr;  // reaction coefficient c = alpha det J at the WQ points [Nq], or none
};

constexpr int kXstageSmemMax = 227 * 1024;

// y = K~ x, y = K~^T x, g6 = dJ/dC (Algorithm 2 and its transpose).  A nonzero
// *skip (device flag, may be NULL) turns every launch into a no-op.
template <typename T>
int run_apply(const OpCtx<T>& c, const T* x, T* y, const int* skip);
template <typename T>
int run_apply_T(const OpCtx<T>& c, const T* x, T* y, const int* skip);
template <typename T>
int run_grad(const OpCtx<T>& c, const T* lam, const T* u, T* g6);
// gc = dJ/dc of the reaction coefficient (Algorithm 1's D)
template <typename T>
int run_grad_mass(const OpCtx<T>& c, const T* lam, const T* u, T* gc);
int mass_smem_bytes(int elem_size, int n1, int nq1);

size_t apply_scratch_elems(const int n[3], const int nq[3]);
size_t rhs_scratch_elems(const int n[3], const int ng[3]);
int xstage_smem_bytes(int elem_size, int n1, int nq1, int lines, int mode);  // forward x stage
bool xstage_mode_valid(int elem_size, int n1, int nq1, int lines, int mode);
int xstage_aux_smem_bytes(int elem_size, int n1, int nq1);         // transposed and gradient x stages
int configure_xstage_smem(int bytes);

int run_eval_coeff(const int nq[3], const double* const xq[3], int geom, const double* modes, int nmodes, double kscale,
                   double* C, cudaStream_t s);
int run_load_vector(const DirD<double> d[3], int geom, int forcing, double* scratch, double* f, cudaStream_t s);
int run_eval_mass(const int nq[3], const double* const xq[3], int geom, double alpha, double* c, cudaStream_t s);
// Relative H1 error against an exact solution (MFWQ_EXACT_*); allocates its
// temporaries, synchronises the stream.
int run_h1_error(const DirD<double> d[3], int geom, int sol, const double* u, double* rel, cudaStream_t s);

// FD preconditioner, FP64: z = P^-1 r; tmp holds N doubles.  skip as above.
int run_fd64(const DirD<double> d[3], const double* r, double* z, double* tmp, const int* skip, cudaStream_t s);
// FD preconditioner in FP32 storage on the FP32 pipe.
int run_fd32_simt(const DirD<float> d[3], const float* r, float* z, float* tmp, const int* skip, cudaStream_t s);
// FD preconditioner on the tensor cores (tcgen05), TF32 or BF16 inputs, FP32
// in/out; every n_l <= 256.  A bounded wait that times out sets *err = 1.
int run_fd_tc(const DirD<float> d[3], int fd_precision, const float* r, float* z, float* tmp, int* err, const int* skip,
              cudaStream_t s);
int configure_fd_tc(int max_n);

}  // namespace mfwq
