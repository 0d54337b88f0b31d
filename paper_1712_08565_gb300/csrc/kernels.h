// Kernel launchers shared by the C-ABI layer (internal).
#pragma once

#include <cuda_runtime.h>

#include "mfwq_internal.h"

namespace mfwq {

struct FusedPlan;  // fused_apply.h

// Coefficient evaluated at the quadrature points inside the FP32 x stage
// instead of read from a stored copy (the memory-lean form of Section 3.2's
// remark on storing C).  K(x) = exp(kscale g(x)) I with the Fourier field
// g(x) = sum_m a_m cos(2 pi k_m . x + phi_m), x = F(xi) the exact map.  For
// both geometries C = |det J| J^-1 K J^-T = kappa(x) G(xi1): G depends on xi1
// only (ring: G = diag(pi r / 2, 2 / (pi r), pi r / 2), r = 1 + xi1; cube:
// G = I), so G is a table over the direction-1 points and only kappa is
// evaluated per point.  With s = r (ring) or xi1 (cube), the phase in
// half-turns is 2 k.x + phi/pi = (2 A) s + B, where A and B depend on the
// line (xi2, xi3) only: ring A = k1 cos(pi xi2 / 2) + k2 sin(pi xi2 / 2),
// B = 2 k3 xi3 + phi/pi; cube A = k1, B = 2 (k2 xi2 + k3 xi3) + phi/pi.
constexpr int kMaxModes = 32;
struct CoeffField {
    int geom = 0;          // MFWQ_GEOM_*
    int nmodes = 0;
    float kscale = 0.f;
    float a[kMaxModes];            // amplitudes
    double k[kMaxModes][3];        // wave vectors
    double phi_pi[kMaxModes];      // phases / pi
    const float* g6 = nullptr;     // [6][nq1]: G at the direction-1 points, fields 11, 22, 33, 12, 13, 23
    const float* s1 = nullptr;     // [2][nq1]: s at the direction-1 points as an unevaluated sum hi + lo
    const double* xq2 = nullptr;   // points of directions 2 and 3
    const double* xq3 = nullptr;
};

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
    int svec = 1;      // FP32 forward slow stages: columns per thread (1, 2 or 4; vector loads and stores)
    int* err = nullptr;  // device error word: set when a bounded wait times out
    const T* cm = nullptr;  // reaction coefficient c = alpha det J at the WQ points [Nq], or none
    const FusedPlan* fused = nullptr;  // FP32: plan of the fused apply (used when ok and no reaction term)
    const CoeffField* cf = nullptr;    // FP32: coefficient evaluated in the x stage (C unused), or none
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
int xstage_otf_smem_bytes(int n1, int nq1);                         // FP32 stencil x stage with the coefficient evaluated
int configure_xstage_otf_smem(int bytes);
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
