// MF-WQ operator kernels for sm_103a: the sum-factorised stiffness apply of
// Algorithm 2 (Section 3.2), its transpose, the coefficient gradient, and the
// setup helpers (coefficient and load vector at the quadrature points).
//
// The apply of K~ = sum_ab W^(ab) D^(ab) B^(b) is split into five banded
// mode-product stages on tensors stored [dim3][dim2][dim1] (dim1 fastest):
//   trial z : v            -> Z0 = B0_3 v, Z1 = B1_3 v                 [nq3][n2][n1]
//   trial y : Z0, Z1       -> Y00, Y10, Y01                             [nq3][nq2][n1]
//   x stage : Y, C         -> T^(ab) = W1^(ab) (C_ab (B_1 Y))  (9)      [nq3][nq2][n1]
//   test y  : T (9)        -> U_z (4, grouped by the z-family)          [nq3][n2][n1]
//   test z  : U (4)        -> w                                         [n3][n2][n1]
// The x stage fuses the last trial contraction, the pointwise product with
// the six coefficient fields and the first test contraction in shared memory,
// so the quadrature-point gradients G_b = B^(b) v never reach HBM.
//
// Index conventions: (alpha, beta) pairs are numbered k = 3(alpha-1) + (beta-1)
// (11,12,13,21,22,23,31,32,33); a 1D weight family (a, b) has index 2a+b; the
// direction-l family of W^(ab) is (a_l, b_l) = ([l=alpha], [l=beta]).
#include <cuda_runtime.h>

#include "kernels.h"
#include "prof.h"

namespace mfwq {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
struct Ptr9 {
    T* p[9];
};

// ---------------------------------------------------------------- slow-dimension band contraction
// out[a][r][c] = sum_t band(r, t) in[a][start(r) + t][c] for the middle (A > 1)
// or the slowest (A = 1) dimension; the Op decides inputs, outputs, families.
struct SlowGeom {
    int A, Rin, Rout, C;
};

template <class Op>
__global__ void __launch_bounds__(kThreads) k_slow(Op op, SlowGeom g, const int* skip) {
    if (skip && *skip) return;
    const int r = blockIdx.y;
    const int s = op.band.start[r];
    const int L = op.band.len[r];
    const size_t AC = (size_t)g.A * g.C;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < AC; e += (size_t)gridDim.x * blockDim.x) {
        const size_t a = e / g.C, c = e - a * g.C;
        const size_t i0 = (a * g.Rin + s) * g.C + c;
        const size_t o = (a * g.Rout + r) * g.C + c;
        op.run(r, L, i0, (size_t)g.C, o);
    }
}

template <typename T>
struct OpTrialZ {  // Z0 = B0 v, Z1 = B1 v
    BandD<T> band;
    const T* __restrict__ v;
    T* __restrict__ z0;
    T* __restrict__ z1;
    __device__ void run(int r, int L, size_t i0, size_t st, size_t o) const {
        const T* b0 = band.row(0, r);
        const T* b1 = band.row(1, r);
        T a0 = 0, a1 = 0;
        for (int t = 0; t < L; ++t) {
            T x = v[i0 + t * st];
            a0 = fmaT(b0[t], x, a0);
            a1 = fmaT(b1[t], x, a1);
        }
        z0[o] = a0;
        z1[o] = a1;
    }
};

template <typename T>
struct OpTrialY {  // Y00 = B0 Z0, Y10 = B1 Z0, Y01 = B0 Z1
    BandD<T> band;
    const T* __restrict__ z0;
    const T* __restrict__ z1;
    T* __restrict__ y00;
    T* __restrict__ y10;
    T* __restrict__ y01;
    __device__ void run(int r, int L, size_t i0, size_t st, size_t o) const {
        const T* b0 = band.row(0, r);
        const T* b1 = band.row(1, r);
        T a = 0, b = 0, c = 0;
        for (int t = 0; t < L; ++t) {
            T x0 = z0[i0 + t * st], x1 = z1[i0 + t * st];
            a = fmaT(b0[t], x0, a);
            b = fmaT(b1[t], x0, b);
            c = fmaT(b0[t], x1, c);
        }
        y00[o] = a;
        y10[o] = b;
        y01[o] = c;
    }
};

template <typename T>
struct OpTestY {  // 9 x-contracted tensors -> 4 z-groups through W2
    BandD<T> band;
    const T* __restrict__ in[9];
    T* __restrict__ out[4];
    __device__ void run(int r, int L, size_t i0, size_t st, size_t o) const {
        const T* w00 = band.row(0, r);
        const T* w01 = band.row(1, r);
        const T* w10 = band.row(2, r);
        const T* w11 = band.row(3, r);
        T u0 = 0, u1 = 0, u2 = 0, u3 = 0;
        for (int t = 0; t < L; ++t) {
            const size_t i = i0 + t * st;
            const T f00 = w00[t], f01 = w01[t], f10 = w10[t], f11 = w11[t];
            // z-family (0,0): pairs 11, 12, 21, 22 with y-families (0,0), (0,1), (1,0), (1,1)
            u0 = fmaT(f00, in[0][i], u0);
            u0 = fmaT(f01, in[1][i], u0);
            u0 = fmaT(f10, in[3][i], u0);
            u0 = fmaT(f11, in[4][i], u0);
            // z-family (0,1): pairs 13 (y 00), 23 (y 10)
            u1 = fmaT(f00, in[2][i], u1);
            u1 = fmaT(f10, in[5][i], u1);
            // z-family (1,0): pairs 31 (y 00), 32 (y 01)
            u2 = fmaT(f00, in[6][i], u2);
            u2 = fmaT(f01, in[7][i], u2);
            // z-family (1,1): pair 33 (y 00)
            u3 = fmaT(f00, in[8][i], u3);
        }
        out[0][o] = u0;
        out[1][o] = u1;
        out[2][o] = u2;
        out[3][o] = u3;
    }
};

template <typename T>
struct OpTestZ {  // w = sum_f W3^f U_f
    BandD<T> band;
    const T* __restrict__ in[4];
    T* __restrict__ out;
    __device__ void run(int r, int L, size_t i0, size_t st, size_t o) const {
        const T* w0 = band.row(0, r);
        const T* w1 = band.row(1, r);
        const T* w2 = band.row(2, r);
        const T* w3 = band.row(3, r);
        T acc = 0;
        for (int t = 0; t < L; ++t) {
            const size_t i = i0 + t * st;
            acc = fmaT(w0[t], in[0][i], acc);
            acc = fmaT(w1[t], in[1][i], acc);
            acc = fmaT(w2[t], in[2][i], acc);
            acc = fmaT(w3[t], in[3][i], acc);
        }
        out[o] = acc;
    }
};

// ---- transposed stages
template <typename T>
struct OpTestZT {  // V_f = W3^f^T y  (band rows q3 -> i3)
    BandD<T> band;
    const T* __restrict__ in;
    T* __restrict__ out[4];
    __device__ void run(int r, int L, size_t i0, size_t st, size_t o) const {
        const T* w0 = band.row(0, r);
        const T* w1 = band.row(1, r);
        const T* w2 = band.row(2, r);
        const T* w3 = band.row(3, r);
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        for (int t = 0; t < L; ++t) {
            T x = in[i0 + t * st];
            a0 = fmaT(w0[t], x, a0);
            a1 = fmaT(w1[t], x, a1);
            a2 = fmaT(w2[t], x, a2);
            a3 = fmaT(w3[t], x, a3);
        }
        out[0][o] = a0;
        out[1][o] = a1;
        out[2][o] = a2;
        out[3][o] = a3;
    }
};

template <typename T>
struct OpTestYT {  // R^(ab) = W2^(y-fam)^T V_(z-fam), 9 outputs
    BandD<T> band;
    const T* __restrict__ in[4];
    T* __restrict__ out[9];
    __device__ void run(int r, int L, size_t i0, size_t st, size_t o) const {
        const T* w00 = band.row(0, r);
        const T* w01 = band.row(1, r);
        const T* w10 = band.row(2, r);
        const T* w11 = band.row(3, r);
        T r11 = 0, r12 = 0, r13 = 0, r21 = 0, r22 = 0, r23 = 0, r31 = 0, r32 = 0, r33 = 0;
        for (int t = 0; t < L; ++t) {
            const size_t i = i0 + t * st;
            const T v0 = in[0][i], v1 = in[1][i], v2 = in[2][i], v3 = in[3][i];
            const T f00 = w00[t], f01 = w01[t], f10 = w10[t], f11 = w11[t];
            r11 = fmaT(f00, v0, r11);
            r12 = fmaT(f01, v0, r12);
            r21 = fmaT(f10, v0, r21);
            r22 = fmaT(f11, v0, r22);
            r13 = fmaT(f00, v1, r13);
            r23 = fmaT(f10, v1, r23);
            r31 = fmaT(f00, v2, r31);
            r32 = fmaT(f01, v2, r32);
            r33 = fmaT(f00, v3, r33);
        }
        out[0][o] = r11;
        out[1][o] = r12;
        out[2][o] = r13;
        out[3][o] = r21;
        out[4][o] = r22;
        out[5][o] = r23;
        out[6][o] = r31;
        out[7][o] = r32;
        out[8][o] = r33;
    }
};

template <typename T>
struct OpTrialYT {  // Zt0 = B0^T X1 + B1^T X2, Zt1 = B0^T X3 (band rows j2 -> q2)
    BandD<T> band;
    const T* __restrict__ x1;
    const T* __restrict__ x2;
    const T* __restrict__ x3;
    T* __restrict__ z0;
    T* __restrict__ z1;
    __device__ void run(int r, int L, size_t i0, size_t st, size_t o) const {
        const T* b0 = band.row(0, r);
        const T* b1 = band.row(1, r);
        T a = 0, b = 0;
        for (int t = 0; t < L; ++t) {
            const size_t i = i0 + t * st;
            a = fmaT(b0[t], x1[i], a);
            a = fmaT(b1[t], x2[i], a);
            b = fmaT(b0[t], x3[i], b);
        }
        z0[o] = a;
        z1[o] = b;
    }
};

template <typename T>
struct OpTrialZT {  // out = B0^T Zt0 + B1^T Zt1 (band rows j3 -> q3)
    BandD<T> band;
    const T* __restrict__ z0;
    const T* __restrict__ z1;
    T* __restrict__ out;
    __device__ void run(int r, int L, size_t i0, size_t st, size_t o) const {
        const T* b0 = band.row(0, r);
        const T* b1 = band.row(1, r);
        T a = 0;
        for (int t = 0; t < L; ++t) {
            const size_t i = i0 + t * st;
            a = fmaT(b0[t], z0[i], a);
            a = fmaT(b1[t], z1[i], a);
        }
        out[o] = a;
    }
};

template <typename T>
struct OpSingle {  // out = band(fam 0) applied to one input (load-vector stages)
    BandD<T> band;
    const T* __restrict__ in;
    T* __restrict__ out;
    __device__ void run(int r, int L, size_t i0, size_t st, size_t o) const {
        const T* b = band.row(0, r);
        T a = 0;
        for (int t = 0; t < L; ++t) a = fmaT(b[t], in[i0 + t * st], a);
        out[o] = a;
    }
};

template <class Op>
cudaError_t launch_slow(int tag, const Op& op, int A, int Rin, int Rout, int C, const int* skip, cudaStream_t s) {
    SlowGeom g{A, Rin, Rout, C};
    size_t AC = (size_t)A * C;
    unsigned bx = (unsigned)((AC + kThreads - 1) / kThreads);
    if (bx > 65535u) bx = 65535u;
    dim3 grid(bx, Rout);
    launch_begin(tag, s);
    k_slow<<<grid, kThreads, 0, s>>>(op, g, skip);
    launch_end(tag, s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- x stage (dim 1, fused)
template <typename T>
struct XArgs {
    BandD<T> B;    // rows q1 -> j1
    BandD<T> BT;   // rows j1 -> q1
    BandD<T> W;    // rows i1 -> q1
    BandD<T> WT;   // rows q1 -> i1
    int n1, nq1, nlines;
    size_t Nq;     // points per coefficient field
    const T* C;    // [6][Nq]
};

constexpr int kLines = 4;

// Forward x stage: Y (3 inputs [line][n1]) -> T (9 outputs [line][n1]).
// The nine products are formed three at a time, one trial direction beta at a
// time: G_b on the lines' points (B1 in direction 1 for beta = 1, else B0),
// H^(ab) = C_ab G_b for alpha = 1..3 in shared memory, then the three test
// contractions with W1^(a1,b1).  Two work mappings (chosen by the autotuner):
//  MODE 0: a thread owns one (line, point) or one (alpha, line, i) item
//          (most items in flight; best for the FP64 pipe);
//  MODE 1: a thread owns one point or one (alpha, i) output for all LINES
//          lines, so each band coefficient it loads serves LINES multiply-adds
//          (fewest loads; best when the FP32 pipe leaves the loads exposed).
template <typename T, int LINES, int MODE>
__global__ void __launch_bounds__(kThreads) k_xstage_apply(XArgs<T> a, const T* __restrict__ y0, const T* __restrict__ y1,
                                                           const T* __restrict__ y2, T* __restrict__ tout, size_t tstride,
                                                           const int* skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    T* sY = reinterpret_cast<T*>(smem_raw);  // [3][LINES][n1]
    T* sH = sY + 3 * LINES * a.n1;           // [3][LINES][nq1]
    const int line0 = blockIdx.x * LINES;
    const int nl = min(LINES, a.nlines - line0);
    const int n1 = a.n1, nq1 = a.nq1;
    const int hs = LINES * nq1;
    for (int e = threadIdx.x; e < nl * n1; e += blockDim.x) {
        const int l = e / n1, j = e - l * n1;
        const size_t gi = (size_t)(line0 + l) * n1 + j;
        sY[(0 * LINES + l) * n1 + j] = y0[gi];
        sY[(1 * LINES + l) * n1 + j] = y1[gi];
        sY[(2 * LINES + l) * n1 + j] = y2[gi];
    }
    for (int b = 0; b < 3; ++b) {
        __syncthreads();
        const int bfam = b == 0 ? 1 : 0;
        // symmetric-storage slots of C_(alpha,beta), alpha = 1..3: alpha if alpha = beta, else 2 + alpha + beta
        const size_t c0 = (size_t)(b == 0 ? 0 : 2 + b) * a.Nq;
        const size_t c1 = (size_t)(b == 1 ? 1 : 3 + b) * a.Nq;
        const size_t c2 = (size_t)(b == 2 ? 2 : 4 + b) * a.Nq;
        if (MODE == 0) {
            for (int e = threadIdx.x; e < nl * nq1; e += blockDim.x) {
                const int l = e / nq1, q = e - l * nq1;
                const int s = a.B.start[q], L = a.B.len[q];
                const T* Y = sY + (b * LINES + l) * n1 + s;
                T g = 0;
                for (int t = 0; t < L; ++t) g = fmaT(a.B.lane(bfam, q, t), Y[t], g);
                const size_t pt = (size_t)(line0 + l) * nq1 + q;
                T* H = sH + l * nq1 + q;
                H[0 * hs] = a.C[c0 + pt] * g;
                H[1 * hs] = a.C[c1 + pt] * g;
                H[2 * hs] = a.C[c2 + pt] * g;
            }
        } else {
            for (int q = threadIdx.x; q < nq1; q += blockDim.x) {
                const int s = a.B.start[q], L = a.B.len[q];
                T g[LINES];
#pragma unroll
                for (int l = 0; l < LINES; ++l) g[l] = 0;
                const T* Y = sY + (b * LINES) * n1 + s;
                for (int t = 0; t < L; ++t) {
                    const T bt = a.B.lane(bfam, q, t);
#pragma unroll
                    for (int l = 0; l < LINES; ++l) g[l] = fmaT(bt, Y[l * n1 + t], g[l]);
                }
#pragma unroll
                for (int l = 0; l < LINES; ++l) {
                    if (l >= nl) break;
                    const size_t pt = (size_t)(line0 + l) * nq1 + q;
                    T* H = sH + l * nq1 + q;
                    H[0 * hs] = a.C[c0 + pt] * g[l];
                    H[1 * hs] = a.C[c1 + pt] * g[l];
                    H[2 * hs] = a.C[c2 + pt] * g[l];
                }
            }
        }
        __syncthreads();
        // outputs; x-family (a1, b1) = ([alpha = 1], [beta = 1])
        if (MODE == 0) {
            const int per = nl * n1;
            for (int e = threadIdx.x; e < 3 * per; e += blockDim.x) {
                const int al = e / per, rem = e - al * per;
                const int l = rem / n1, i = rem - l * n1;
                const int fam = 2 * (al == 0 ? 1 : 0) + bfam;
                const int s = a.W.start[i], L = a.W.len[i];
                const T* H = sH + (al * LINES + l) * nq1 + s;
                T acc = 0;
                for (int t = 0; t < L; ++t) acc = fmaT(a.W.lane(fam, i, t), H[t], acc);
                tout[(size_t)(3 * al + b) * tstride + (size_t)(line0 + l) * n1 + i] = acc;
            }
        } else {
            for (int e = threadIdx.x; e < 3 * n1; e += blockDim.x) {
                const int al = e / n1, i = e - al * n1;
                const int fam = 2 * (al == 0 ? 1 : 0) + bfam;
                const int s = a.W.start[i], L = a.W.len[i];
                const T* H = sH + (al * LINES) * nq1 + s;
                T acc[LINES];
#pragma unroll
                for (int l = 0; l < LINES; ++l) acc[l] = 0;
                for (int t = 0; t < L; ++t) {
                    const T wt = a.W.lane(fam, i, t);
#pragma unroll
                    for (int l = 0; l < LINES; ++l) acc[l] = fmaT(wt, H[l * nq1 + t], acc[l]);
                }
                T* o = tout + (size_t)(3 * al + b) * tstride + (size_t)line0 * n1 + i;
#pragma unroll
                for (int l = 0; l < LINES; ++l) {
                    if (l >= nl) break;
                    o[(size_t)l * n1] = acc[l];
                }
            }
        }
    }
}

template <typename T, int MODE>
void launch_xstage(int L, dim3 grid, size_t sm, cudaStream_t st, const XArgs<T>& a, const T* y0, const T* y1, const T* y2,
                   T* tout, size_t tstride, const int* skip) {
    if (L == 2) k_xstage_apply<T, 2, MODE><<<grid, kThreads, sm, st>>>(a, y0, y1, y2, tout, tstride, skip);
    else if (L == 8) k_xstage_apply<T, 8, MODE><<<grid, kThreads, sm, st>>>(a, y0, y1, y2, tout, tstride, skip);
    else k_xstage_apply<T, 4, MODE><<<grid, kThreads, sm, st>>>(a, y0, y1, y2, tout, tstride, skip);
}

// Transposed x stage: R (9 inputs [line][n1]) -> S^(ab) = W1^T R at q1 ->
// E_b = sum_a C_ab S^(ab) -> X_b = B1^(b)T E_b (3 outputs [line][n1]).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_xstage_applyT(XArgs<T> a, Ptr9<T> rin,
                                                            T* __restrict__ x1, T* __restrict__ x2, T* __restrict__ x3,
                                                            const int* skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    T* sR = reinterpret_cast<T*>(smem_raw);  // [9][kLines][n1]
    T* sE = sR + 9 * kLines * a.n1;          // [3][kLines][nq1]
    const int line0 = blockIdx.x * kLines;
    const int nl = min(kLines, a.nlines - line0);
    const int n1 = a.n1, nq1 = a.nq1;
    for (int e = threadIdx.x; e < nl * n1; e += blockDim.x) {
        const int l = e / n1, j = e - l * n1;
        const size_t gi = (size_t)(line0 + l) * n1 + j;
#pragma unroll
        for (int k = 0; k < 9; ++k) sR[(k * kLines + l) * n1 + j] = rin.p[k][gi];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nl * nq1; e += blockDim.x) {
        const int l = e / nq1, q = e - l * nq1;
        const int s = a.WT.start[q], L = a.WT.len[q];
        const int fs = kLines * n1;
        const T* R = sR + l * n1 + s;
        T S[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) S[k] = 0;
        for (int t = 0; t < L; ++t) {
            const T f00 = a.WT.lane(0, q, t), f01 = a.WT.lane(1, q, t), f10 = a.WT.lane(2, q, t), f11 = a.WT.lane(3, q, t);
            S[0] = fmaT(f11, R[0 * fs + t], S[0]);
            S[1] = fmaT(f10, R[1 * fs + t], S[1]);
            S[2] = fmaT(f10, R[2 * fs + t], S[2]);
            S[3] = fmaT(f01, R[3 * fs + t], S[3]);
            S[4] = fmaT(f00, R[4 * fs + t], S[4]);
            S[5] = fmaT(f00, R[5 * fs + t], S[5]);
            S[6] = fmaT(f01, R[6 * fs + t], S[6]);
            S[7] = fmaT(f00, R[7 * fs + t], S[7]);
            S[8] = fmaT(f00, R[8 * fs + t], S[8]);
        }
        const size_t pt = (size_t)(line0 + l) * nq1 + q;
        const T c11 = a.C[pt], c22 = a.C[a.Nq + pt], c33 = a.C[2 * a.Nq + pt];
        const T c12 = a.C[3 * a.Nq + pt], c13 = a.C[4 * a.Nq + pt], c23 = a.C[5 * a.Nq + pt];
        const int es = kLines * nq1;
        T* E = sE + l * nq1 + q;
        E[0 * es] = c11 * S[0] + c12 * S[3] + c13 * S[6];  // beta = 1: C_11 S11 + C_21 S21 + C_31 S31
        E[1 * es] = c12 * S[1] + c22 * S[4] + c23 * S[7];  // beta = 2
        E[2 * es] = c13 * S[2] + c23 * S[5] + c33 * S[8];  // beta = 3
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nl * n1; e += blockDim.x) {
        const int l = e / n1, j = e - l * n1;
        const int s = a.BT.start[j], L = a.BT.len[j];
        const int es = kLines * nq1;
        const T* E = sE + l * nq1 + s;
        T o1 = 0, o2 = 0, o3 = 0;
        for (int t = 0; t < L; ++t) {
            const T b0 = a.BT.lane(0, j, t), b1 = a.BT.lane(1, j, t);
            o1 = fmaT(b1, E[0 * es + t], o1);
            o2 = fmaT(b0, E[1 * es + t], o2);
            o3 = fmaT(b0, E[2 * es + t], o3);
        }
        const size_t go = (size_t)(line0 + l) * n1 + j;
        x1[go] = o1;
        x2[go] = o2;
        x3[go] = o3;
    }
}

// Gradient x stage: G_b from Y (trial partials of u), S^(ab) from R (test
// partials of lambda); g_ab = -S^(ab) G_b folded into 6 symmetric slots.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_xstage_grad(XArgs<T> a, const T* __restrict__ y0, const T* __restrict__ y1,
                                                          const T* __restrict__ y2, Ptr9<T> rin, T* __restrict__ g6) {
    extern __shared__ unsigned char smem_raw[];
    T* sY = reinterpret_cast<T*>(smem_raw);  // [3][kLines][n1]
    T* sR = sY + 3 * kLines * a.n1;          // [9][kLines][n1]
    const int line0 = blockIdx.x * kLines;
    const int nl = min(kLines, a.nlines - line0);
    const int n1 = a.n1, nq1 = a.nq1;
    for (int e = threadIdx.x; e < nl * n1; e += blockDim.x) {
        const int l = e / n1, j = e - l * n1;
        const size_t gi = (size_t)(line0 + l) * n1 + j;
        sY[(0 * kLines + l) * n1 + j] = y0[gi];
        sY[(1 * kLines + l) * n1 + j] = y1[gi];
        sY[(2 * kLines + l) * n1 + j] = y2[gi];
#pragma unroll
        for (int k = 0; k < 9; ++k) sR[(k * kLines + l) * n1 + j] = rin.p[k][gi];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nl * nq1; e += blockDim.x) {
        const int l = e / nq1, q = e - l * nq1;
        const int fs = kLines * n1;
        T g1 = 0, g2 = 0, g3 = 0;
        {
            const int s = a.B.start[q], L = a.B.len[q];
            const T* Y = sY + l * n1 + s;
            for (int t = 0; t < L; ++t) {
                const T b0 = a.B.lane(0, q, t), b1 = a.B.lane(1, q, t);
                g1 = fmaT(b1, Y[0 * fs + t], g1);
                g2 = fmaT(b0, Y[1 * fs + t], g2);
                g3 = fmaT(b0, Y[2 * fs + t], g3);
            }
        }
        T S[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) S[k] = 0;
        {
            const int s = a.WT.start[q], L = a.WT.len[q];
            const T* R = sR + l * n1 + s;
            for (int t = 0; t < L; ++t) {
                const T f00 = a.WT.lane(0, q, t), f01 = a.WT.lane(1, q, t), f10 = a.WT.lane(2, q, t), f11 = a.WT.lane(3, q, t);
                S[0] = fmaT(f11, R[0 * fs + t], S[0]);
                S[1] = fmaT(f10, R[1 * fs + t], S[1]);
                S[2] = fmaT(f10, R[2 * fs + t], S[2]);
                S[3] = fmaT(f01, R[3 * fs + t], S[3]);
                S[4] = fmaT(f00, R[4 * fs + t], S[4]);
                S[5] = fmaT(f00, R[5 * fs + t], S[5]);
                S[6] = fmaT(f01, R[6 * fs + t], S[6]);
                S[7] = fmaT(f00, R[7 * fs + t], S[7]);
                S[8] = fmaT(f00, R[8 * fs + t], S[8]);
            }
        }
        const size_t pt = (size_t)(line0 + l) * nq1 + q;
        g6[pt] = -S[0] * g1;
        g6[a.Nq + pt] = -S[4] * g2;
        g6[2 * a.Nq + pt] = -S[8] * g3;
        g6[3 * a.Nq + pt] = -(S[1] * g2 + S[3] * g1);
        g6[4 * a.Nq + pt] = -(S[2] * g3 + S[6] * g1);
        g6[5 * a.Nq + pt] = -(S[5] * g3 + S[7] * g2);
    }
}

template <typename T>
XArgs<T> xargs(const DirD<T>& d1, int nlines, size_t Nq, const T* C) {
    XArgs<T> a;
    a.B = d1.B;
    a.BT = d1.BT;
    a.W = d1.W;
    a.WT = d1.WT;
    a.n1 = d1.n;
    a.nq1 = d1.nq;
    a.nlines = nlines;
    a.Nq = Nq;
    a.C = C;
    return a;
}

// ---------------------------------------------------------------- geometry
__device__ void geometry_at(int geom, double xi1, double xi2, double xi3, double X[3], double J[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] = 0.0;
    if (geom == MFWQ_GEOM_RING) {
        const double hp = 1.5707963267948966;  // pi / 2
        const double r = 1.0 + xi1;
        double sn, cs;
        sincos(hp * xi2, &sn, &cs);
        X[0] = r * cs;
        X[1] = r * sn;
        X[2] = xi3;
        J[0][0] = cs;
        J[1][0] = sn;
        J[0][1] = -r * hp * sn;
        J[1][1] = r * hp * cs;
        J[2][2] = 1.0;
    } else {
        X[0] = xi1;
        X[1] = xi2;
        X[2] = xi3;
        J[0][0] = J[1][1] = J[2][2] = 1.0;
    }
}

struct Modes {
    int n;
    double kscale;
    double m[32][5];
};

__device__ double kappa_at(const Modes& md, const double X[3]) {
    if (md.n == 0) return 1.0;
    const double twopi = 6.283185307179586;
    double g = 0.0;
    for (int i = 0; i < md.n; ++i)
        g += md.m[i][0] * cos(twopi * (md.m[i][1] * X[0] + md.m[i][2] * X[1] + md.m[i][3] * X[2]) + md.m[i][4]);
    return exp(md.kscale * g);
}

// C = |det J| kappa J^-1 J^-T at every WQ point.
__global__ void k_eval_coeff(int geom, Modes md, const double* __restrict__ xq1, const double* __restrict__ xq2,
                             const double* __restrict__ xq3, int nq1, int nq2, int nq3, double* __restrict__ C) {
    const size_t Nq = (size_t)nq1 * nq2 * nq3;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < Nq; p += (size_t)gridDim.x * blockDim.x) {
        const int q1 = (int)(p % nq1);
        const int q2 = (int)((p / nq1) % nq2);
        const int q3 = (int)(p / ((size_t)nq1 * nq2));
        double X[3], J[3][3];
        geometry_at(geom, xq1[q1], xq2[q2], xq3[q3], X, J);
        // adjugate inverse
        double A[3][3];
        A[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        A[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        A[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        A[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        A[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        A[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        A[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        A[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        A[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double det = J[0][0] * A[0][0] + J[0][1] * A[1][0] + J[0][2] * A[2][0];
        // J^-1 = A / det;  C = |det| kappa J^-1 J^-T = kappa A A^T / |det|
        const double f = kappa_at(md, X) / fabs(det);
        const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
        for (int s = 0; s < 6; ++s) {
            const int i = pr[s][0], j = pr[s][1];
            C[s * Nq + p] = f * (A[i][0] * A[j][0] + A[i][1] * A[j][1] + A[i][2] * A[j][2]);
        }
    }
}

__device__ double forcing_at(int forcing, const double X[3]) {
    const double pi = 3.141592653589793;
    if (forcing == MFWQ_FORCING_RING_EXACT) {
        const double k = 5.0 * pi;
        double s1, c1, s2, c2, s3, c3;
        sincos(k * X[0], &s1, &c1);
        sincos(k * X[1], &s2, &c2);
        sincos(k * X[2], &s3, &c3);
        const double rho = X[0] * X[0] + X[1] * X[1];
        const double q = (rho - 1.0) * (rho - 4.0);
        const double S = s1 * s2 * s3;
        const double lapS = -3.0 * k * k * S;
        const double gsq = (2.0 * rho - 5.0) * 2.0 * (X[0] * k * c1 * s2 * s3 + X[1] * k * s1 * c2 * s3);
        const double lapq = 8.0 * rho + (2.0 * rho - 5.0) * 4.0;
        return -(q * lapS + 2.0 * gsq + S * lapq);
    }
    return 3.0 * pi * pi * sin(pi * X[0]) * sin(pi * X[1]) * sin(pi * X[2]);
}

// Load vector, x stage: out[g3][g2][j1] = sum_g1 GT1[j1] |det J| f(F(xi)) on
// each Gauss line (g3, g2); the Gauss weights sit in the GT bands.
__global__ void __launch_bounds__(kThreads) k_rhs_x(int geom, int forcing, BandD<double> GT1, const double* __restrict__ xg1,
                                                    const double* __restrict__ xg2, const double* __restrict__ xg3,
                                                    int ng1, int ng2, int n1, double* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    double* sF = reinterpret_cast<double*>(smem_raw);  // [ng1]
    const int line = blockIdx.x;
    const int g2 = line % ng2, g3 = line / ng2;
    for (int g = threadIdx.x; g < ng1; g += blockDim.x) {
        double X[3], J[3][3];
        geometry_at(geom, xg1[g], xg2[g2], xg3[g3], X, J);
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        sF[g] = fabs(det) * forcing_at(forcing, X);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n1; j += blockDim.x) {
        const int s = GT1.start[j], L = GT1.len[j];
        double acc = 0.0;
        for (int t = 0; t < L; ++t) acc = fmaT(GT1.lane(0, j, t), sF[s + t], acc);
        out[(size_t)line * n1 + j] = acc;
    }
}

}  // namespace

// ================================================================= host launchers
template <typename T>
int run_apply(const OpCtx<T>& c, const T* x, T* y, const int* skip) {
    const DirD<T>& d1 = c.d[0];
    const DirD<T>& d2 = c.d[1];
    const DirD<T>& d3 = c.d[2];
    const int n1 = d1.n, n2 = d2.n, n3 = d3.n, q1 = d1.nq, q2 = d2.nq, q3 = d3.nq;
    const size_t SP = (size_t)q3 * q2 * n1, SQ = (size_t)q3 * n2 * n1;
    T* P = c.scratch;           // 12 x SP
    T* Q = c.scratch + 12 * SP; // 4 x SQ
    T* Z0 = Q;
    T* Z1 = Q + SQ;
    T* Y[3] = {P, P + SP, P + 2 * SP};
    T* Tt[9];
    for (int k = 0; k < 9; ++k) Tt[k] = P + (3 + k) * SP;
    cudaError_t e;
    // trial z
    OpTrialZ<T> oz{d3.B, x, Z0, Z1};
    if ((e = launch_slow(S_TRIAL_Z, oz, 1, n3, q3, n2 * n1, skip, c.stream)) != cudaSuccess) return MFWQ_ECUDA;
    // trial y
    OpTrialY<T> oy{d2.B, Z0, Z1, Y[0], Y[1], Y[2]};
    if ((e = launch_slow(S_TRIAL_Y, oy, q3, n2, q2, n1, skip, c.stream)) != cudaSuccess) return MFWQ_ECUDA;
    // x stage (lines per block chosen by the autotuner: 2, 4 or 8)
    {
        XArgs<T> a = xargs(d1, q3 * q2, c.Nq, c.C);
        const int L = c.xlines == 2 || c.xlines == 8 ? c.xlines : 4;
        size_t sm = sizeof(T) * ((size_t)3 * L * n1 + (size_t)3 * L * q1);
        dim3 grid((q3 * q2 + L - 1) / L);
        launch_begin(S_XSTAGE, c.stream);
        if (c.xmode == 1) launch_xstage<T, 1>(L, grid, sm, c.stream, a, Y[0], Y[1], Y[2], Tt[0], SP, skip);
        else launch_xstage<T, 0>(L, grid, sm, c.stream, a, Y[0], Y[1], Y[2], Tt[0], SP, skip);
        launch_end(S_XSTAGE, c.stream);
        if (cudaGetLastError() != cudaSuccess) return MFWQ_ECUDA;
    }
    // test y: 9 -> 4 (U reuses Q)
    OpTestY<T> oty;
    oty.band = d2.W;
    for (int k = 0; k < 9; ++k) oty.in[k] = Tt[k];
    for (int f = 0; f < 4; ++f) oty.out[f] = Q + f * SQ;
    if ((e = launch_slow(S_TEST_Y, oty, q3, q2, n2, n1, skip, c.stream)) != cudaSuccess) return MFWQ_ECUDA;
    // test z
    OpTestZ<T> otz;
    otz.band = d3.W;
    for (int f = 0; f < 4; ++f) otz.in[f] = Q + f * SQ;
    otz.out = y;
    if ((e = launch_slow(S_TEST_Z, otz, 1, q3, n3, n2 * n1, skip, c.stream)) != cudaSuccess) return MFWQ_ECUDA;
    return MFWQ_OK;
}

// Transposed test side of lambda: V (4, in Q) and R (9, in P[3..12)).
template <typename T>
static int run_test_T_partials(const OpCtx<T>& c, const T* x, const int* skip) {
    const DirD<T>& d2 = c.d[1];
    const DirD<T>& d3 = c.d[2];
    const int n1 = c.d[0].n, n2 = d2.n, n3 = d3.n, q2 = d2.nq, q3 = d3.nq;
    const size_t SP = (size_t)q3 * q2 * n1, SQ = (size_t)q3 * n2 * n1;
    T* P = c.scratch;
    T* Q = c.scratch + 12 * SP;
    OpTestZT<T> o1;
    o1.band = d3.WT;
    o1.in = x;
    for (int f = 0; f < 4; ++f) o1.out[f] = Q + f * SQ;
    if (launch_slow(S_TEST_ZT, o1, 1, n3, q3, n2 * n1, skip, c.stream) != cudaSuccess) return MFWQ_ECUDA;
    OpTestYT<T> o2;
    o2.band = d2.WT;
    for (int f = 0; f < 4; ++f) o2.in[f] = Q + f * SQ;
    for (int k = 0; k < 9; ++k) o2.out[k] = P + (3 + k) * SP;
    if (launch_slow(S_TEST_YT, o2, q3, n2, q2, n1, skip, c.stream) != cudaSuccess) return MFWQ_ECUDA;
    return MFWQ_OK;
}

template <typename T>
int run_apply_T(const OpCtx<T>& c, const T* x, T* y, const int* skip) {
    const DirD<T>& d1 = c.d[0];
    const DirD<T>& d2 = c.d[1];
    const DirD<T>& d3 = c.d[2];
    const int n1 = d1.n, n2 = d2.n, n3 = d3.n, q1 = d1.nq, q2 = d2.nq, q3 = d3.nq;
    const size_t SP = (size_t)q3 * q2 * n1, SQ = (size_t)q3 * n2 * n1;
    T* P = c.scratch;
    T* Q = c.scratch + 12 * SP;
    int st = run_test_T_partials(c, x, skip);
    if (st != MFWQ_OK) return st;
    // x stage: R (P[3..12)) -> X1, X2, X3 (P[0..3))
    {
        XArgs<T> a = xargs(d1, q3 * q2, c.Nq, c.C);
        size_t sm = sizeof(T) * ((size_t)9 * kLines * n1 + (size_t)3 * kLines * q1);
        dim3 grid((q3 * q2 + kLines - 1) / kLines);
        Ptr9<T> rp;
        for (int k = 0; k < 9; ++k) rp.p[k] = P + (3 + k) * SP;
        launch_begin(S_XSTAGE_T, c.stream);
        k_xstage_applyT<T><<<grid, kThreads, sm, c.stream>>>(a, rp, P, P + SP, P + 2 * SP, skip);
        launch_end(S_XSTAGE_T, c.stream);
        if (cudaGetLastError() != cudaSuccess) return MFWQ_ECUDA;
    }
    OpTrialYT<T> o3{d2.BT, P, P + SP, P + 2 * SP, Q, Q + SQ};
    if (launch_slow(S_TRIAL_YT, o3, q3, q2, n2, n1, skip, c.stream) != cudaSuccess) return MFWQ_ECUDA;
    OpTrialZT<T> o4{d3.BT, Q, Q + SQ, y};
    if (launch_slow(S_TRIAL_ZT, o4, 1, q3, n3, n2 * n1, skip, c.stream) != cudaSuccess) return MFWQ_ECUDA;
    return MFWQ_OK;
}

template <typename T>
int run_grad(const OpCtx<T>& c, const T* lam, const T* u, T* g6) {
    const DirD<T>& d1 = c.d[0];
    const DirD<T>& d2 = c.d[1];
    const DirD<T>& d3 = c.d[2];
    const int n1 = d1.n, n2 = d2.n, n3 = d3.n, q2 = d2.nq, q3 = d3.nq;
    const size_t SP = (size_t)q3 * q2 * n1, SQ = (size_t)q3 * n2 * n1;
    T* P = c.scratch;
    T* Q = c.scratch + 12 * SP;
    // trial partials of u: Z (Q[0..2)) -> Y (P[0..3))
    OpTrialZ<T> oz{d3.B, u, Q, Q + SQ};
    if (launch_slow(S_TRIAL_Z, oz, 1, n3, q3, n2 * n1, nullptr, c.stream) != cudaSuccess) return MFWQ_ECUDA;
    OpTrialY<T> oy{d2.B, Q, Q + SQ, P, P + SP, P + 2 * SP};
    if (launch_slow(S_TRIAL_Y, oy, q3, n2, q2, n1, nullptr, c.stream) != cudaSuccess) return MFWQ_ECUDA;
    // test partials of lambda: V (Q) -> R (P[3..12))
    int st = run_test_T_partials(c, lam, nullptr);
    if (st != MFWQ_OK) return st;
    XArgs<T> a = xargs(d1, q3 * q2, c.Nq, c.C);
    size_t sm = sizeof(T) * ((size_t)12 * kLines * n1);
    dim3 grid((q3 * q2 + kLines - 1) / kLines);
    Ptr9<T> rp;
    for (int k = 0; k < 9; ++k) rp.p[k] = P + (3 + k) * SP;
    launch_begin(S_XSTAGE_GRAD, c.stream);
    k_xstage_grad<T><<<grid, kThreads, sm, c.stream>>>(a, P, P + SP, P + 2 * SP, rp, g6);
    launch_end(S_XSTAGE_GRAD, c.stream);
    if (cudaGetLastError() != cudaSuccess) return MFWQ_ECUDA;
    (void)n3;
    return MFWQ_OK;
}

size_t apply_scratch_elems(const int n[3], const int nq[3]) {
    return 12 * (size_t)nq[2] * nq[1] * n[0] + 4 * (size_t)nq[2] * n[1] * n[0];
}

size_t rhs_scratch_elems(const int n[3], const int ng[3]) {
    return (size_t)ng[2] * ng[1] * n[0] + (size_t)ng[2] * n[1] * n[0];
}

int xstage_smem_bytes(int elem_size, int n1, int nq1, int lines) {
    return (int)(((size_t)3 * lines * n1 + (size_t)3 * lines * nq1) * elem_size);
}

int xstage_aux_smem_bytes(int elem_size, int n1, int nq1) {
    size_t b = (size_t)9 * kLines * n1 + (size_t)3 * kLines * nq1;  // transposed x stage
    size_t c = (size_t)12 * kLines * n1;                             // gradient x stage
    return (int)((b > c ? b : c) * elem_size);
}

// The dynamic shared-memory limit is a per-kernel attribute shared by all
// handles, so it only ever grows.
int configure_xstage_smem(int bytes) {
    static int configured = 0;
    if (bytes <= configured) return MFWQ_OK;
    cudaError_t e = cudaSuccess;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    e = cudaFuncSetAttribute(k_xstage_apply<double, 2, 0>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<double, 4, 0>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<double, 8, 0>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<float, 2, 0>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<float, 4, 0>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<float, 8, 0>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<double, 2, 1>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<double, 4, 1>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<double, 8, 1>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<float, 2, 1>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<float, 4, 1>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_apply<float, 8, 1>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_applyT<double>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_grad<double>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_applyT<float>, A, bytes);
    if (e == cudaSuccess) configured = bytes;
    return e == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}

int run_eval_coeff(const int nq[3], const double* const xq[3], int geom, const double* modes, int nmodes, double kscale,
                   double* C, cudaStream_t s) {
    Modes md;
    md.n = nmodes;
    md.kscale = kscale;
    for (int i = 0; i < nmodes; ++i)
        for (int j = 0; j < 5; ++j) md.m[i][j] = modes[i * 5 + j];
    size_t Nq = (size_t)nq[0] * nq[1] * nq[2];
    unsigned blocks = (unsigned)((Nq + 255) / 256);
    if (blocks > 65535u * 8u) blocks = 65535u * 8u;
    launch_begin(S_SETUP, s);
    k_eval_coeff<<<blocks, 256, 0, s>>>(geom, md, xq[0], xq[1], xq[2], nq[0], nq[1], nq[2], C);
    launch_end(S_SETUP, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}

int run_load_vector(const DirD<double> d[3], int geom, int forcing, double* scratch, double* f, cudaStream_t s) {
    const int n1 = d[0].n, n2 = d[1].n, n3 = d[2].n, g1 = d[0].ng, g2 = d[1].ng, g3 = d[2].ng;
    double* A = scratch;                                // [g3][g2][n1]
    double* B = scratch + (size_t)g3 * g2 * n1;         // [g3][n2][n1]
    size_t sm = sizeof(double) * (size_t)g1;
    launch_begin(S_SETUP, s);
    k_rhs_x<<<g3 * g2, kThreads, sm, s>>>(geom, forcing, d[0].GT, d[0].xg, d[1].xg, d[2].xg, g1, g2, n1, A);
    launch_end(S_SETUP, s);
    if (cudaGetLastError() != cudaSuccess) return MFWQ_ECUDA;
    OpSingle<double> oy{d[1].GT, A, B};
    if (launch_slow(S_SETUP, oy, g3, g2, n2, n1, nullptr, s) != cudaSuccess) return MFWQ_ECUDA;
    OpSingle<double> oz{d[2].GT, B, f};
    if (launch_slow(S_SETUP, oz, 1, g3, n3, n2 * n1, nullptr, s) != cudaSuccess) return MFWQ_ECUDA;
    return MFWQ_OK;
}

template int run_apply<double>(const OpCtx<double>&, const double*, double*, const int*);
template int run_apply<float>(const OpCtx<float>&, const float*, float*, const int*);
template int run_apply_T<double>(const OpCtx<double>&, const double*, double*, const int*);
template int run_grad<double>(const OpCtx<double>&, const double*, const double*, double*);

}  // namespace mfwq
