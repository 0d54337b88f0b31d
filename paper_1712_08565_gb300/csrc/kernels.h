// Kernel launchers shared by the C-ABI layer (internal).
#pragma once

#include <cuda_runtime.h>

#include "mfwq_internal.h"

namespace mfwq {

// Everything one operator application needs, in one precision.
template <typename T>
struct OpCtx {
    DirD<T> d[3];
    const T* C;        // [6][Nq]
    size_t Nq;
    T* scratch;        // apply_scratch_elems() elements of T
    cudaStream_t stream;
    int xlines = 4;    // (q3, q2) lines per block of the forward x stage: 2, 4 or 8
    int xmode = 0;     // forward x-stage work mapping: 0 per (line, item), 1 per item over all lines
};

// y = K~ x, y = K~^T x, g6 = dJ/dC (Algorithm 2 and its transpose).  A nonzero
// *skip (device flag, may be NULL) turns every launch into a no-op.
template <typename T>
int run_apply(const OpCtx<T>& c, const T* x, T* y, const int* skip);
template <typename T>
int run_apply_T(const OpCtx<T>& c, const T* x, T* y, const int* skip);
template <typename T>
int run_grad(const OpCtx<T>& c, const T* lam, const T* u, T* g6);

size_t apply_scratch_elems(const int n[3], const int nq[3]);
size_t rhs_scratch_elems(const int n[3], const int ng[3]);
int xstage_smem_bytes(int elem_size, int n1, int nq1, int lines);  // forward x stage
int xstage_aux_smem_bytes(int elem_size, int n1, int nq1);         // transposed and gradient x stages
int configure_xstage_smem(int bytes);

int run_eval_coeff(const int nq[3], const double* const xq[3], int geom, const double* modes, int nmodes, double kscale,
                   double* C, cudaStream_t s);
int run_load_vector(const DirD<double> d[3], int geom, int forcing, double* scratch, double* f, cudaStream_t s);

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
