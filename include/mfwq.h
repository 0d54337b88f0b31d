/*
 * mfwq.h -- C ABI of the GB300 (sm_103a) matrix-free weighted-quadrature
 * (MF-WQ) isogeometric k-method library.
 *
 * The operator is the weighted-quadrature stiffness of Sangalli & Tani,
 * "Matrix-free weighted quadrature for a computationally efficient
 * isogeometric k-method", applied matrix-free through the factorisation
 *     K~ = sum_{alpha,beta=1..3} W^(alpha,beta) D^(alpha,beta) B^(beta)
 * of Section 3.2 (Algorithm 2), preconditioned by the Fast Diagonalization
 * (FD) method and solved with BiCGStab (Section 4).
 *
 * Conventions shared by every call
 *  - Tensors of degrees of freedom (DoFs) have n1*n2*n3 entries stored as a
 *    C array [i3][i2][i1] (direction 1 fastest, Eq. (ordering) and the scalar
 *    index of Section 2.1).  Quadrature-point tensors have nq1*nq2*nq3 entries
 *    stored [q3][q2][q1].  n_l = (number of B-splines in direction l) - 2
 *    (homogeneous Dirichlet, Section 2.1); nq_l = 2*nel_l + 2*p_l - 1 (the WQ
 *    point rule of Section 2.2: every interior knot, every interior-span
 *    midpoint, p+1 equispaced points inside the first and the last span).
 *  - The symmetric coefficient C = |det J| J^-1 K J^-T (Eq. (C), J_ij =
 *    dF_i/dxi_j) is stored as 6 fields [6][nq3][nq2][nq1] in the order
 *    C11, C22, C33, C12, C13, C23 (Section 3.2: d(d+1)/2 fields suffice).
 *  - Pointers named *_dev are device pointers owned by the caller, at least
 *    16-byte aligned; input and output buffers of one call must not overlap.
 *    Pointers named *_host are host pointers.
 *  - Work is enqueued on the stream given at setup.  Calls documented as
 *    "asynchronous" return after enqueueing; launch errors are reported at
 *    once, and nothing else can fail on the device.  Calls documented as
 *    "synchronous" wait for the stream.
 *  - Every call returns an MFWQ_* status; nothing aborts, traps or throws.
 *  - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef MFWQ_H
#define MFWQ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define MFWQ_OK          0
#define MFWQ_EINVAL     -1  /* bad argument: size, degree, knot vector, NULL, alignment */
#define MFWQ_ENOMEM     -2  /* a device or host allocation failed */
#define MFWQ_ECUDA      -3  /* a CUDA runtime call or kernel launch failed */
#define MFWQ_ESETUP     -4  /* a weight system was inconsistent or an eigensolve failed */
#define MFWQ_EBREAKDOWN -5  /* BiCGStab breakdown: rho, r^.v or omega vanished */
#define MFWQ_ENOCONV    -6  /* the solve did not reach rtol within maxit */
#define MFWQ_ETIMEOUT   -7  /* a bounded device-side wait gave up */
#define MFWQ_ENAN       -8  /* a NaN or Inf appeared in a Krylov scalar */
#define MFWQ_EINTERNAL  -9

/* ---- enumerations -------------------------------------------------------- */
#define MFWQ_FD_FP64 0  /* FD mode products in FP64 (FP64 pipe) */
#define MFWQ_FD_TF32 1  /* FD mode products on tensor cores, TF32 inputs, FP32 accumulate */
#define MFWQ_FD_BF16 2  /* FD mode products on tensor cores, BF16 inputs, FP32 accumulate */

#define MFWQ_GEOM_CUBE 0  /* F = identity on [0,1]^3 */
#define MFWQ_GEOM_RING 1  /* thick quarter ring of Section 4, exact polar map
                             F(xi) = ((1+xi1) cos(pi xi2/2), (1+xi1) sin(pi xi2/2), xi3) */

#define MFWQ_FORCING_SINES      0  /* f = 3 pi^2 sin(pi x1) sin(pi x2) sin(pi x3) */
#define MFWQ_FORCING_RING_EXACT 1  /* f = -Laplace u for Eq. (exact-solution) */

typedef struct mfwq_handle_s* mfwq_handle;

/* ---- setup --------------------------------------------------------------- */
typedef struct {
    int degree[3];            /* p_l >= 2, <= 12 (C^{p-1} splines, Section 2.1) */
    int nknots[3];            /* length of knots[l] = nel_l + 2 p_l + 1 */
    const double* knots[3];   /* host; open knot vector on [0,1]: p+1 zeros, strictly
                                 increasing interior knots (multiplicity 1), p+1 ones */
    int mixed;                /* 0: FP64 operator and FP64 FD only.
                                 1: also build the FP32 operator and the tensor-core FD
                                 used by the mixed-precision refinement of mfwq_solve. */
    int fd_precision;         /* FD precision of the mixed inner solve: MFWQ_FD_TF32 or
                                 MFWQ_FD_BF16 (ignored when mixed = 0) */
    void* stream;             /* cudaStream_t all work is enqueued on (NULL = legacy) */
} mfwq_setup_desc;

/* Builds the 1D tables of Algorithm 2's setup on the host (B-spline values and
 * derivatives at the WQ points, Eq. (Bl); the four weight families per
 * direction, Eq. (exactness1d)/(exactness_K)/(weights-support) solved in the
 * minimum-2-norm sense; the FD factors U_l, lambda_l of the generalized
 * eigenproblem K_l U = M_l U Lambda), uploads them and allocates the handle's
 * device workspace.  The coefficient must then be given with mfwq_set_coeff.
 * Returns MFWQ_EINVAL for a bad descriptor, MFWQ_ESETUP if a weight system is
 * inconsistent, MFWQ_ENOMEM / MFWQ_ECUDA on device failures.  Synchronous. */
int mfwq_setup(const mfwq_setup_desc* desc, mfwq_handle* out);

/* Frees everything the handle owns.  NULL is allowed. */
void mfwq_destroy(mfwq_handle h);

/* Static text for a status code. */
const char* mfwq_status_string(int status);

/* Message describing the last failure of a call made from this thread (empty
 * if none).  The pointer stays valid until the next failing call. */
const char* mfwq_last_error(void);

/* n[l] = DoFs and nq[l] = WQ points in direction l (either may be NULL). */
int mfwq_sizes(mfwq_handle h, int n[3], int nq[3]);

/* WQ points of direction dir (0, 1, 2) into xq_host[nq[dir]]. */
int mfwq_quad_points(mfwq_handle h, int dir, double* xq_host);

/* Host-only (no CUDA call): the 1D tables for one direction, dense, for
 * inspection and tests.  Pass NULL for any output not wanted; *n and *nq are
 * always written.  xq[nq]; B0, B1 [nq][n] (row q, column j); W [4][n][nq]
 * with family index 2a+b of the pair (a, b) (a: derivative order of the test
 * function, b: of the trial function); U [n][n] (column k = k-th eigenvector,
 * U^T M U = I) and lam[n] of the FD factorisation. */
int mfwq_tables_1d(int degree, int nknots, const double* knots, int* n, int* nq,
                   double* xq, double* B0, double* B1, double* W, double* U, double* lam);

/* ---- coefficient and right-hand side (setup helpers, not the hot path) ---- */
/* C_dev[6][nq3][nq2][nq1] = C at the WQ points for the given geometry and
 * K(x) = exp(kscale * g(x)) I, g(x) = sum_m a_m cos(2 pi k_m . x + phi_m) in
 * physical coordinates.  modes_host holds nmodes rows (a, k1, k2, k3, phi)
 * (nmodes <= 32; nmodes = 0 gives K = I).  Asynchronous. */
int mfwq_eval_coeff(mfwq_handle h, int geometry, const double* modes_host, int nmodes,
                    double kscale, double* C_dev);

/* Copies C_dev[6][Nq] into the handle (and an FP32 copy when mixed).  The
 * caller's buffer may be reused afterwards.  Turns off a coefficient
 * evaluated in the FP32 operator (mfwq_set_coeff_field).  Asynchronous. */
int mfwq_set_coeff(mfwq_handle h, const double* C_dev);

/* Sets the coefficient from its definition: C = |det J| J^-1 K J^-T (Eq. (C))
 * for the given geometry and K(x) = exp(kscale g(x)) I, g as in
 * mfwq_eval_coeff (modes_host: nmodes rows (a, k1, k2, k3, phi), nmodes <= 32).
 * The FP64 coefficient is evaluated and stored as by mfwq_eval_coeff followed
 * by mfwq_set_coeff.  With onthefly = 1 (mixed handles) the FP32 operator does
 * not store C at all: its x stage evaluates C at every quadrature point from
 * the map and the field, the memory-lean form of the paper's remark on
 * storing the coefficient (Section 3.2), and the 6 Nq FP32 values are freed.
 * Both geometries give C = kappa(x) G(xi1), with G = |det J| J^-1 J^-T a
 * function of xi1 alone, so G is a table over the direction-1 points and
 * kappa = exp(kscale g(F(xi))) is computed per point in FP32 (CUDA's cospif and
 * expf, phase reduced modulo one period before rounding).  onthefly = 1 needs
 * the stencil form of the x stage (p_1 <= 8) and makes the FP32 operator use
 * it.  MFWQ_EINVAL on a bad argument or an unsupported handle.  Synchronous. */
int mfwq_set_coeff_field(mfwq_handle h, int geometry, const double* modes_host, int nmodes, double kscale,
                         int onthefly);

/* ---- reaction (mass) term: alpha u in Eq. (poisson) ----------------------
 * The discrete operator becomes K~ + M~ with the WQ mass matrix of Eq. (Mwq),
 * M~_ij = sum_q w_iq c(x_q) b_j(x_q), c = alpha det J (Eq. (M)), applied
 * matrix-free as M~ = W D B (Algorithm 1, Section 3.1) inside every apply,
 * transposed apply and solve of the handle (FP64 and, on a mixed handle,
 * FP32).  The weights are the (0,0) family of the stiffness weights in every
 * direction. */

/* c_dev[nq3][nq2][nq1] = alpha |det J| at the WQ points for the given
 * geometry and a constant alpha.  Asynchronous. */
int mfwq_eval_mass_coeff(mfwq_handle h, int geometry, double alpha, double* c_dev);

/* Copies c_dev[Nq] (c at the WQ points, any real values) into the handle and
 * turns the reaction term on; c_dev = NULL turns it off and frees the copy.
 * fd_shift (finite, >= 0) is added to every eigenvalue sum of the FD
 * preconditioner, which then inverts P + fd_shift M3 (x) M2 (x) M1 exactly
 * (same eigenvectors); a constant alpha on a cube-like patch suggests
 * fd_shift = alpha.  The paper gives no preconditioner for alpha > 0.
 * MFWQ_EINVAL on a negative or non-finite shift.  Asynchronous. */
int mfwq_set_mass_coeff(mfwq_handle h, const double* c_dev, double fd_shift);

/* Load vector f_i = int |det J| b_i (f o F) dxi (Eq. (linearsystem)) by
 * tensor Gauss quadrature with p+1 points per span.  Asynchronous. */
int mfwq_load_vector(mfwq_handle h, int geometry, int forcing, double* f_dev);

/* ---- error measure of Section 4 (post-processing, not the hot path) ------- */
enum {
    MFWQ_EXACT_SINES = 0,  /* u = sin(pi x) sin(pi y) sin(pi z): the cube with MFWQ_FORCING_SINES */
    MFWQ_EXACT_RING = 1    /* Eq. (exact-solution) on the ring, MFWQ_FORCING_RING_EXACT */
};

/* *rel_err (host) = ||u - u_h||_H1 / ||u||_H1 for the discrete function with
 * coefficients u_dev[n3][n2][n1] against the exact solution, by tensor Gauss
 * quadrature with p_l + 2 points per span, physical gradients J^-T grad_xi.
 * The Gauss-point values are formed by sum factorisation in slabs of about
 * 0.5 GB (allocated and freed by the call).  MFWQ_ENOMEM if that fails.
 * Synchronous. */
int mfwq_h1_error(mfwq_handle h, int geometry, int solution, const double* u_dev, double* rel_err);

/* ---- hot path ------------------------------------------------------------ */
/* y = K~ x, FP64 (Algorithm 2, sum-factorised).  x_dev, y_dev: [n3][n2][n1].
 * Uses the handle's workspace, so calls on one handle must not overlap on the
 * device.  Asynchronous. */
int mfwq_apply(mfwq_handle h, const double* x_dev, double* y_dev);

/* y = K~^T x = sum B^(beta)^T D^(alpha,beta) W^(alpha,beta)^T x, FP64 (the WQ
 * matrix is not symmetric, Section 4).  Asynchronous. */
int mfwq_apply_T(mfwq_handle h, const double* x_dev, double* y_dev);

/* y = K~ x in FP32 (FP32 tables and coefficient; needs mixed = 1). */
int mfwq_apply_f32(mfwq_handle h, const float* x_dev, float* y_dev);

/* z = P^-1 r, FD preconditioner in FP64: P = M3(x)M2(x)K1 + M3(x)K2(x)M1 +
 * K3(x)M2(x)M1, P^-1 = (U3(x)U2(x)U1) diag(1/(l1_i+l2_j+l3_k)) (U3(x)U2(x)U1)^T.
 * Asynchronous. */
int fd_precond(mfwq_handle h, const double* r_dev, double* z_dev);

/* z = P^-1 r in the handle's low precision (TF32 or BF16 tensor-core mode
 * products, FP32 accumulate, FP32 in and out; needs mixed = 1). */
int fd_precond_f32(mfwq_handle h, const float* r_dev, float* z_dev);

/* The FP32 operator of a mixed handle runs in one of two kernel sequences
 * that compute the same Algorithm 2 (results agree to FP32 rounding):
 *  MFWQ_PATH_STAGED: five kernels, one banded contraction direction each (the
 *    x stage fusing the trial x contraction, the coefficient product and the
 *    test x contraction), partial tensors passed through device memory;
 *  MFWQ_PATH_FUSED: trial z, then one kernel for the trial y contraction, the
 *    x stage and the test y contraction per (q3 plane, run of q2 lines), with
 *    the y partials kept on chip, then test z.  Available where the stencil
 *    form of the x stage is (p_1 <= 8); not used while a reaction term is on.
 * The staged path is the default; mfwq_autotune times both and keeps the faster.
 * mfwq_set_fp32_path returns MFWQ_EINVAL (reason in mfwq_last_error) for
 * MFWQ_PATH_FUSED where it is unavailable; mfwq_fp32_path returns the path in
 * use.  Neither launches work. */
#define MFWQ_PATH_STAGED 0
#define MFWQ_PATH_FUSED 1
int mfwq_set_fp32_path(mfwq_handle h, int path);
int mfwq_fp32_path(mfwq_handle h);

/* Kernels of the FP64 FD preconditioner (fd_precond and the FP64 solves):
 *  MFWQ_FD64_PIPE: the mode products in FP64 on the FP64 pipe (even/odd
 *    split where the knot vectors are symmetric); the default where a
 *    direction has more than 256 DoFs;
 *  MFWQ_FD64_SPLIT: the mode products on the BF16 tensor cores, every FP64
 *    operand split into 8 integer slices of 7 bits under a power-of-two scale
 *    per row (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012); the
 *    slice products accumulate exactly, and the result keeps 56 bits below
 *    each row's leading power of two, so it agrees with the FP64 products to
 *    about 2^-55 of sum |U_ij| |x_j|.  Needs every n_l <= 256, and is then
 *    the default: mfwq_setup slices the mode matrices and allocates N
 *    doubles for the eigenvalue scaling and about 17 bytes per DoF of slice
 *    workspace.
 * mfwq_set_fd64_path returns MFWQ_EINVAL for an unknown path or sizes above
 * 256; mfwq_fd64_path returns the path in use. */
#define MFWQ_FD64_PIPE 0
#define MFWQ_FD64_SPLIT 1
int mfwq_set_fd64_path(mfwq_handle h, int path);
int mfwq_fd64_path(mfwq_handle h);

/* Thread tiling of the four slow-dimension stages (the z and y contractions
 * of Algorithm 2): each thread computes `rows` consecutive output rows (1, 2
 * or 4) of `cols` consecutive columns (1, 2 or 4; FP32 forward stages only,
 * loaded and stored as one 8- or 16-byte vector; a stage whose column count
 * or buffers are not aligned to it runs one column per thread).  fp32 = 0
 * sets the FP64 operator (cols must be 1), 1 the FP32 operator of a mixed
 * handle.  Every output is summed in the same order under every tiling, so
 * the results are bitwise the same; mfwq_autotune sets both by timing.
 * Returns MFWQ_EINVAL for other values; launches no work.  mfwq_slow_tiling
 * writes the tiling in use to *rows and *cols. */
int mfwq_set_slow_tiling(mfwq_handle h, int fp32, int rows, int cols);
int mfwq_slow_tiling(mfwq_handle h, int fp32, int* rows, int* cols);

typedef struct {
    double rtol;           /* stop when ||f - K~ u||_2 <= rtol ||f||_2 */
    int maxit;             /* BiCGStab iterations (outer refinement steps when mixed) */
    double inner_rtol;     /* mixed: relative tolerance of each inner FP32 solve (0: 1e-4) */
    int inner_maxit;       /* mixed: iteration cap of each inner solve (0: 200) */
    int use_initial_guess; /* 0: start from u = 0; 1: u_dev holds the initial guess */
    int force_fp64;        /* 1: plain FP64 solve even on a mixed handle */
    double* res_hist;      /* host, may be NULL: relative residual after each iteration
                              (maxit + 1 entries) */
    int fp64_low_fd;       /* 1 (mixed handle, single patch): FP64 BiCGStab as with force_fp64,
                              with the FD applied in the handle's low precision (FP64 -> FP32,
                              tensor-core mode products, FP32 -> FP64).  The iterate, the
                              operator and the residual stay FP64, so the tolerance is met in
                              FP64; only the preconditioner is inexact.  MFWQ_EINVAL on a
                              handle without mixed = 1 and in mfwq_batch_solve. */
    int graph_chunk;       /* FP64 single-patch solves: > 1 captures that many BiCGStab iterations
                              into one CUDA graph, launched between two host checks of the
                              device-resident scalars (iterations after convergence are skipped
                              on the device); 0 or 1: one check per iteration.  Ignored with
                              res_hist, while profiling, on the legacy stream, and when the
                              capture fails (the iterations then run uncaptured). */
} mfwq_solve_opts;

typedef struct {
    int status;            /* MFWQ_OK, MFWQ_ENOCONV, MFWQ_EBREAKDOWN, MFWQ_ENAN */
    int iterations;        /* BiCGStab iterations (summed over inner solves when mixed) */
    int outer_iterations;  /* refinement steps (mixed), else 0 */
    double rel_residual;   /* last ||f - K~ u|| / ||f|| (FP64 residual) */
} mfwq_solve_info;

/* Solves K~ u = f with right-FD-preconditioned BiCGStab (Section 4): FP64
 * throughout, or -- on a mixed handle -- FP64 iterative refinement around
 * inner FP32 BiCGStab solves (FP32 operator, tensor-core FD, FP32 vector
 * updates, dot products taken per thread by the compensated Dot2 scheme in
 * FP32 and summed across threads in FP64).  f_dev, u_dev: [n3][n2][n1].
 * Synchronous; returns info->status. */
int mfwq_solve(mfwq_handle h, const double* f_dev, double* u_dev,
               const mfwq_solve_opts* opts, mfwq_solve_info* info);

/* Solves the adjoint system K~^T lambda = g (FD is symmetric, so the same
 * preconditioner serves).  FP64.  Synchronous. */
int mfwq_solve_T(mfwq_handle h, const double* g_dev, double* lambda_dev,
                 const mfwq_solve_opts* opts, mfwq_solve_info* info);

/* mfwq_solve with host buffers: copies f_host to the device, solves, copies
 * u back into u_host (both [n3][n2][n1]).  Synchronous. */
int mfwq_solve_host(mfwq_handle h, const double* f_host, double* u_host,
                    const mfwq_solve_opts* opts, mfwq_solve_info* info);

/* Gradient of J with respect to the stored coefficient fields, given the
 * state u (K~ u = f) and the adjoint lambda (K~^T lambda = dJ/du).  Because
 * K~ is linear in every C_ab(x_q) (Section 3.2),
 *   dJ/dC_ab(q) = -(W^(ab)^T lambda)_q (B^(b) u)_q,
 * and the symmetric slot of an off-diagonal pair receives the sum of both
 * orderings.  gC_dev: [6][nq3][nq2][nq1].  The quadrature-point gradients
 * B^(b) u are recomputed, not stored.  Asynchronous. */
int mfwq_grad_coeff(mfwq_handle h, const double* lambda_dev, const double* u_dev, double* gC_dev);

/* Gradient of J with respect to the reaction coefficient c at the WQ points:
 * dJ/dc(q) = -(W^T lambda)_q (B u)_q with the mass factors of Algorithm 1.
 * gc_dev: [nq3][nq2][nq1].  Works whether or not the term is on.  Asynchronous. */
int mfwq_grad_mass_coeff(mfwq_handle h, const double* lambda_dev, const double* u_dev, double* gc_dev);

/* Waits for the handle's stream and reports any failure seen since the last call. */
int mfwq_sync(mfwq_handle h);

/* ---- FD preconditioner that allocates nothing -------------------------------
 * No counterpart in the paper: an engineering variant of fd_precond for
 * callers that cannot allocate device memory where they need the
 * preconditioner -- code running while a CUDA graph is captured in global
 * mode (cudaMalloc is illegal then), code whose device memory is all owned by
 * a framework's caching allocator, or code with a fixed memory budget.  It
 * needs no handle: the caller passes the FD factors of each direction (U_l and
 * U_l^T, row-major n_l x n_l, and lambda_l; e.g. from mfwq_tables_1d), the
 * input r and the output z ([n3][n2][n1], FP64, device), and a stream.  The
 * one intermediate tensor lives in a fixed device array of
 * MFWQ_NOALLOC_MAX_N doubles (32 MB) that is part of the library's module, so
 * every GPU that loads the library holds it until the process exits.
 * - n1*n2*n3 > MFWQ_NOALLOC_MAX_N is rejected with MFWQ_EINVAL.
 * - Every pointer (factors, r, z) must be device memory of the calling
 *   thread's current device (or managed memory), and `stream` must belong to
 *   that device: the scratch address is the current device's.  Host memory
 *   and other devices' memory are rejected with MFWQ_EINVAL before any work.
 * - The first call on a device looks the array's address up
 *   (cudaGetSymbolAddress, which may load the module); make that first call
 *   before any stream capture.
 * - Calls share the array: calls whose work overlaps on the GPU (several
 *   streams, several host threads) race and give wrong results.  Each call
 *   overwrites the array completely before reading it, so nothing carries
 *   over from the previous call.
 * - Asynchronous on `stream`; no cudaMalloc/cudaFree or allocating routine. */
#define MFWQ_NOALLOC_MAX_N 4194304
int mfwq_fd_precond_noalloc(const int n[3], const double* const U_dev[3], const double* const UT_dev[3],
                            const double* const lam_dev[3], const double* r_dev, double* z_dev, void* stream);

/* ---- autotuner and batched solve --------------------------------------------
 * No counterpart in the paper (which solves one patch sequentially); multi-patch
 * independence is the uncoupled case of the multi-patch setting the paper
 * names as future work in its conclusions. */

/* Times mfwq_apply (and mfwq_apply_f32 on a mixed handle) on this handle's
 * sizes and keeps the fastest launch shapes: first the forward x stage with 2,
 * 4 and 8 (q3,q2) lines per block and four work mappings (0: one thread per
 * line and item, 1: one thread per item over all lines of the block, 2 and 3:
 * the same with the block's inputs prefetched into shared memory by bulk
 * copies, where the slabs allow it; 4 and 5: 8 lines per block, a thread owns
 * a two-row tile and 4 or 8 lines; each with the default or a reduced
 * shared-memory carveout), then 1, 2 or 4 output rows per thread in the other
 * four stages, and for the FP32 operator the fused kernel sequence
 * (MFWQ_PATH_FUSED, where available) against the best staged one (cached
 * codes add 10000 when the fused one won) and 1, 2 or 4 columns per thread
 * in its slow stages (cached codes add 100000 times the columns when above 1).  *xlines_out (may be NULL) receives the FP64 choice as
 * 1000 * carveout + 100 * rows + 10 * mapping + lines.  cache_path (may be
 * NULL) is a file of JSON lines {"key": "...", "xstage": that code}: a hit
 * skips the timing, a miss appends the result (codes below 100 mean one row
 * per thread).  Uses
 * the handle's Krylov work vectors, so call it between solves.  Synchronous. */
int mfwq_autotune(mfwq_handle h, const char* cache_path, int* xlines_out);

typedef struct mfwq_batch_s* mfwq_batch;

/* A batch of independent patches, each set up (and given its coefficient) as a
 * handle of its own; the handles stay owned by the caller and must outlive the
 * batch.  The batch owns one stream per patch. */
int mfwq_batch_create(int count, const mfwq_handle* patches, mfwq_batch* out);
void mfwq_batch_destroy(mfwq_batch b);

/* Solves K~_i u_i = f_i for every patch.  FP64 form (force_fp64, or any patch
 * without mixed = 1): FD-preconditioned BiCGStab as mfwq_solve, one sweep (a
 * BiCGStab iteration of every patch) per CUDA graph launch; every patch keeps
 * its own device-resident scalars, and a converged patch's work is skipped on
 * the device; outer_iterations holds the number of sweeps.  Two sweep forms
 * (mfwq_batch_set_grouped), with the same results bit for bit:
 *  - per-patch streams (the default): each patch's kernels on a stream of its
 *    own inside the graph, so the patches' stages overlap freely;
 *  - grouped: one persistent launch per kernel stage for a group of patches
 *    (about 55 launches per sweep and group, groups on concurrent streams),
 *    whose blocks walk a device table of the group's work items -- built from
 *    each patch's own launch sequence with its arguments -- and skip converged
 *    patches; the x stage runs in mapping 0 with 4 lines per block.  Needs no
 *    reaction term and the same FD form (even/odd split or not) in every patch;
 *    otherwise the per-patch streams run.
 * Mixed form (every patch mixed = 1): FP64 refinement steps in lockstep over
 * the patches still above rtol, each inner FP32 solve of all of them one graph
 * launch per sweep on per-patch streams; iterations sums a patch's inner
 * iterations, outer_iterations counts its refinement steps.  f_dev[i],
 * u_dev[i]: device vectors of patch i.  infos (count entries, may be NULL)
 * receive each patch's status, iterations and FP64 relative residual.  Returns
 * the first failing patch status (MFWQ_OK if all converged).  Synchronous. */
int mfwq_batch_solve(mfwq_batch b, const double* const* f_dev, double* const* u_dev, const mfwq_solve_opts* opts,
                     mfwq_solve_info* infos);

/* grouped = G > 0 makes the FP64 batched solve run grouped sweeps in G
 * concurrent groups of patches (balanced by size) where they apply; 0 (the
 * default) keeps the per-patch streams.  mfwq_batch_last_grouped returns 1 if
 * the last FP64 batched solve ran grouped sweeps, else 0.  Neither launches
 * work; MFWQ_EINVAL for G < 0. */
int mfwq_batch_set_grouped(mfwq_batch b, int grouped);
int mfwq_batch_last_grouped(mfwq_batch b);

/* ---- self-test of the bounded device waits (no counterpart in the paper) ---
 * Every wait of the library's kernels on an asynchronous copy or MMA is
 * bounded; on timeout the kernel records it in the handle's error word (read
 * by mfwq_sync as MFWQ_ETIMEOUT) and returns.  This call runs that machinery
 * on purpose: one block arms an mbarrier for 16 bytes that no copy delivers
 * and waits at most limit_cycles (1 .. ~4e9 SM cycles) on `stream` (may be
 * NULL).  Returns MFWQ_ETIMEOUT when the wait gave up as designed (the
 * context stays usable), MFWQ_EINTERNAL if it did not.  Synchronous. */
int mfwq_selftest_bounded_wait(long long limit_cycles, void* stream);

/* ---- arithmetic-throughput probe (no counterpart in the paper) ------------
 * *tflops = the fused multiply-add throughput of the current device in FP64
 * (fp64 = 1) or FP32 (fp64 = 0), in TFLOP/s (an FMA counts 2): every thread
 * runs independent FMA chains in registers; the best rate over three timed
 * launches (after one warm-up) at each of 4, 8 and 16 blocks per SM (CUDA
 * events on `stream`, may be NULL).  The measured
 * denominator of the FP64- and FP32-pipe rooflines.  Allocates a small
 * output buffer; changes no device setting.  Synchronous. */
int mfwq_probe_fma_rate(int fp64, void* stream, double* tflops);

/* ---- instrumentation (no counterpart in the paper) -------------------------
 * Kernel stages, in the index order of mfwq_profile_stats: trial_z, trial_y,
 * xstage, test_y, test_z (the five stages of the apply), test_zT, test_yT,
 * xstage_T, trial_yT, trial_zT (the transpose), xstage_grad, fd_dim1,
 * fd_dim23, fd_tc (FD mode products), krylov (BiCGStab vector and scalar
 * kernels), setup, fd_fold (even/odd folding of the FP64 FD), mass (the
 * reaction-term passes), h1_error (mfwq_h1_error), fused_xy (the fused FP32
 * trial-y / x / test-y kernel), fd_oz (FP64 FD mode products on the tensor
 * cores by operand splitting). */
#define MFWQ_NSTAGES 24
typedef struct {
    double ms[MFWQ_NSTAGES];           /* summed device time per stage (CUDA events) */
    long long launches[MFWQ_NSTAGES];  /* kernel launches per stage */
} mfwq_profile_stats;

/* With on = 1, every kernel the handle launches afterwards is bracketed by
 * CUDA events on the handle's stream (a few microseconds per launch). */
int mfwq_profile_enable(mfwq_handle h, int on);

/* Restricts the event bracketing of mfwq_profile_enable to the stages whose
 * bit (1 << stage index) is set in mask (default: all).  Launches of other
 * stages are still counted.  Launches no work. */
int mfwq_profile_stage_mask(mfwq_handle h, unsigned long long mask);

/* Waits for the recorded events and sums them per stage; reset = 1 clears the
 * totals afterwards.  Synchronous. */
int mfwq_profile_read(mfwq_handle h, mfwq_profile_stats* out, int reset);

/* Name of a stage index ("" if out of range). */
const char* mfwq_stage_name(int stage);

/* Kernels launched by the library in this process so far (all handles). */
long long mfwq_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* MFWQ_H */
