// Right-preconditioned BiCGStab (Section 4: BiCGStab for the non-symmetric
// WQ system, FD preconditioner) with every scalar kept on the device.
//
// One iteration (x0 given, r^ = r_0):
//   rho = r^.r, beta = (rho/rho_old)(alpha/omega), p = r + beta (p - omega v)
//   p^ = P^-1 p, v = A p^, alpha = rho / r^.v, s = r - alpha v   [stop if |s| <= tol |f|]
//   s^ = P^-1 s, t = A s^, omega = t.s / t.t
//   x += alpha p^ + omega s^, r = s - omega t                     [stop if |r| <= tol |f|]
// Dot products are reduced deterministically (fixed grid, per-block partial
// sums, one finishing block) and accumulated in FP64; for FP32 vectors each
// thread's part is a Dot2 sum in FP32 (twice-FP32 accuracy, see Dot2F).
// Scalar updates run in one-thread "finish" kernels; the host only reads the
// scalar block to decide when to stop, so the launch sequence of an
// iteration is fixed and the kernels of a finished solve return at once.
#include <cmath>
#include <cuda_runtime.h>

#include "grouped.h"
#include "krylov.h"
#include "prof.h"

namespace mfwq {
namespace {

constexpr int kRedThreads = 256;

template <typename T>
__device__ __forceinline__ double D(T x) { return (double)x; }

__device__ void block_sum2(double& a, double& b, double* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[2 * w] = a;
        sh[2 * w + 1] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sh[2 * lane] : 0.0;
        b = lane < nw ? sh[2 * lane + 1] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// Vector kernels.  Each writes two partial sums per block (part[2 blk], part[2 blk + 1]).
enum { V_INIT = 0, V_P, V_DOT_RV, V_S, V_DOT_TS, V_XR };

template <typename T>
struct VArgs {
    size_t N;
    const T* f;
    T* x;
    T* r;
    T* rhat;
    T* p;
    T* v;
    T* s;
    T* t;
    const T* ph;
    const T* sh;
    int x_given;  // V_INIT: x holds x0 and r = f - A x0 (r preset by the caller)
};

// A dot product's running part in FP32 as the Dot2 algorithm of Ogita, Rump
// and Oishi (Accurate sum and dot product, SIAM J. Sci. Comput. 26, 2005):
// every product split exactly into its rounded value and error (one FMA),
// the rounded values summed with the exact error of each addition (TwoSum)
// kept beside them, so p + s is as accurate as a sum taken in twice the FP32
// precision.  Intrinsics keep the compiler from contracting the error terms.
struct Dot2F {
    float p = 0.f, s = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float h = __fmul_rn(a, b);
        const float r = fmaf(a, b, -h);
        const float x = __fadd_rn(p, h);
        const float z = __fsub_rn(x, p);
        const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(x, z)), __fsub_rn(h, z));
        p = x;
        s = __fadd_rn(s, __fadd_rn(q, r));
    }
    __device__ __forceinline__ double value() const { return (double)p + (double)s; }
};

// FP32 vectors (the inner solve of the mixed-precision refinement): the
// updates in FP32, as an FP32 BiCGStab computes them; each thread's part of a
// dot product by Dot2 in FP32, the block and grid reductions in FP64.  (FP64
// conversions and arithmetic per element would make these memory-streaming
// kernels FP64-pipe bound on this part.)
template <int OP>
__device__ __forceinline__ void vec_f32(const VArgs<float>& a, const KScal* __restrict__ sc, double& s0, double& s1,
                                        int bx, int gdx) {
    const float beta = (float)sc->beta, omega = (float)sc->omega, alpha = (float)sc->alpha;
    const int half = sc->half;
    Dot2F k0, k1;
    for (size_t i = (size_t)bx * blockDim.x + threadIdx.x; i < a.N; i += (size_t)gdx * blockDim.x) {
        if (OP == V_INIT) {
            const float fi = a.f[i];
            const float ri = a.x_given ? a.r[i] : fi;
            if (!a.x_given) a.x[i] = 0.f;
            a.r[i] = ri;
            a.rhat[i] = ri;
            a.p[i] = 0.f;
            a.v[i] = 0.f;
            k0.add(ri, ri);
            k1.add(fi, fi);
        } else if (OP == V_P) {
            a.p[i] = fmaf(beta, fmaf(-omega, a.v[i], a.p[i]), a.r[i]);
        } else if (OP == V_DOT_RV) {
            k0.add(a.rhat[i], a.v[i]);
        } else if (OP == V_S) {
            const float si = fmaf(-alpha, a.v[i], a.r[i]);
            a.s[i] = si;
            k0.add(si, si);
        } else if (OP == V_DOT_TS) {
            const float ti = a.t[i];
            k0.add(ti, a.s[i]);
            k1.add(ti, ti);
        } else if (OP == V_XR) {
            if (half) {
                a.x[i] = fmaf(alpha, a.ph[i], a.x[i]);
            } else {
                a.x[i] = fmaf(omega, a.sh[i], fmaf(alpha, a.ph[i], a.x[i]));
                const float ri = fmaf(-omega, a.t[i], a.s[i]);
                a.r[i] = ri;
                k0.add(ri, ri);
                k1.add(a.rhat[i], ri);
            }
        }
    }
    s0 = k0.value();
    s1 = k1.value();
}

// One block (virtual index bx of gdx) of a vector kernel; sh: 64 doubles of
// shared memory.  Every block writes its two partial sums.
template <typename T, int OP>
__device__ __forceinline__ void vec_body(const VArgs<T>& a, const KScal* __restrict__ sc, double* __restrict__ part,
                                         int bx, int gdx, double* sh) {
    double s0 = 0.0, s1 = 0.0;
    const double beta = sc->beta, omega = sc->omega, alpha = sc->alpha;
    const int half = sc->half;
    if constexpr (sizeof(T) == 4) {
        vec_f32<OP>(a, sc, s0, s1, bx, gdx);
    } else {
        for (size_t i = (size_t)bx * blockDim.x + threadIdx.x; i < a.N; i += (size_t)gdx * blockDim.x) {
            if (OP == V_INIT) {
                T ri = a.x_given ? a.r[i] : a.f[i];
                if (!a.x_given) a.x[i] = 0;
                a.r[i] = ri;
                a.rhat[i] = ri;
                a.p[i] = 0;
                a.v[i] = 0;
                s0 += D(ri) * D(ri);
                s1 += D(a.f[i]) * D(a.f[i]);
            } else if (OP == V_P) {
                a.p[i] = (T)(D(a.r[i]) + beta * (D(a.p[i]) - omega * D(a.v[i])));
            } else if (OP == V_DOT_RV) {
                s0 += D(a.rhat[i]) * D(a.v[i]);
            } else if (OP == V_S) {
                T si = (T)(D(a.r[i]) - alpha * D(a.v[i]));
                a.s[i] = si;
                s0 += D(si) * D(si);
            } else if (OP == V_DOT_TS) {
                s0 += D(a.t[i]) * D(a.s[i]);
                s1 += D(a.t[i]) * D(a.t[i]);
            } else if (OP == V_XR) {
                if (half) {
                    a.x[i] = (T)(D(a.x[i]) + alpha * D(a.ph[i]));
                } else {
                    a.x[i] = (T)(D(a.x[i]) + alpha * D(a.ph[i]) + omega * D(a.sh[i]));
                    T ri = (T)(D(a.s[i]) - omega * D(a.t[i]));
                    a.r[i] = ri;
                    s0 += D(ri) * D(ri);
                    s1 += D(a.rhat[i]) * D(ri);
                }
            }
        }
    }
    if (OP == V_P) return;
    block_sum2(s0, s1, sh);
    if (threadIdx.x == 0) {
        part[2 * bx] = s0;
        part[2 * bx + 1] = s1;
    }
}

template <typename T, int OP>
__global__ void __launch_bounds__(kRedThreads) k_vec(VArgs<T> a, const KScal* __restrict__ sc, double* __restrict__ part) {
    if (OP == V_DOT_TS ? sc->skip2 : sc->skip1) return;
    __shared__ double sh[64];
    vec_body<T, OP>(a, sc, part, blockIdx.x, gridDim.x, sh);
}

__device__ bool finite(double x) { return isfinite(x); }

// Finishing kernels: one block sums the partials in a fixed order, then one
// thread updates the scalars.
template <int OP>
__device__ __forceinline__ void finish_body(KScal* __restrict__ sc, const double* __restrict__ part, int nblk, double* sh) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        s0 += part[2 * i];
        s1 += part[2 * i + 1];
    }
    block_sum2(s0, s1, sh);
    if (threadIdx.x != 0) return;
    if (OP == V_INIT) {
        sc->r2 = s0;
        sc->f2 = s1;
        sc->tol2 = sc->rtol * sc->rtol * s1;
        sc->rho = s0;
        sc->rho_old = sc->alpha = sc->omega = 1.0;
        sc->beta = 0.0;
        sc->iters = 0;
        sc->half = 0;
        sc->status = MFWQ_OK;
        sc->skip1 = sc->skip2 = 0;
        if (!finite(s0) || !finite(s1)) {
            sc->status = MFWQ_ENAN;
            sc->skip1 = sc->skip2 = 1;
        } else if (s1 == 0.0 || s0 <= sc->tol2) {
            sc->skip1 = sc->skip2 = 1;  // already converged (f = 0 gives u = 0)
        }
    } else if (OP == V_DOT_RV) {
        if (!finite(s0)) {
            sc->status = MFWQ_ENAN;
            sc->skip1 = sc->skip2 = 1;
        } else if (s0 == 0.0) {
            sc->status = MFWQ_EBREAKDOWN;
            sc->skip1 = sc->skip2 = 1;
        } else {
            sc->alpha = sc->rho / s0;
        }
    } else if (OP == V_S) {
        sc->s2 = s0;
        if (!finite(s0)) {
            sc->status = MFWQ_ENAN;
            sc->skip1 = sc->skip2 = 1;
        } else if (s0 <= sc->tol2) {
            sc->half = 1;
            sc->skip2 = 1;
        }
    } else if (OP == V_DOT_TS) {
        if (!finite(s0) || !finite(s1)) {
            sc->status = MFWQ_ENAN;
            sc->skip1 = sc->skip2 = 1;
        } else if (s1 == 0.0) {
            sc->status = MFWQ_EBREAKDOWN;
            sc->skip1 = sc->skip2 = 1;
        } else {
            sc->omega = s0 / s1;
        }
    } else if (OP == V_XR) {
        sc->iters += 1;
        if (sc->half) {
            sc->r2 = sc->s2;
            sc->skip1 = sc->skip2 = 1;
            return;
        }
        sc->r2 = s0;
        const double rho_new = s1;
        if (!finite(s0) || !finite(s1)) {
            sc->status = MFWQ_ENAN;
            sc->skip1 = sc->skip2 = 1;
        } else if (s0 <= sc->tol2) {
            sc->skip1 = sc->skip2 = 1;
        } else if (sc->omega == 0.0 || rho_new == 0.0) {
            sc->status = MFWQ_EBREAKDOWN;
            sc->skip1 = sc->skip2 = 1;
        } else {
            sc->rho_old = sc->rho;
            sc->rho = rho_new;
            sc->beta = (sc->rho / sc->rho_old) * (sc->alpha / sc->omega);
        }
    }
}

template <int OP>
__global__ void __launch_bounds__(kRedThreads) k_finish(KScal* __restrict__ sc, const double* __restrict__ part, int nblk) {
    if (OP == V_INIT) {
        // always runs
    } else if (OP == V_DOT_TS ? sc->skip2 : sc->skip1) {
        return;
    }
    __shared__ double sh[64];
    finish_body<OP>(sc, part, nblk, sh);
}

// ---- grouped forms (batched FP64 solve)
struct VecG {
    VArgs<double> a;
    const KScal* sc;
    double* part;
    int nblk;
};
struct FinG {
    KScal* sc;
    const double* part;
    int nblk;
};

template <int OP>
__global__ void __launch_bounds__(kRedThreads) k_vec_grouped(const unsigned char* __restrict__ tab, int stride, int npatch) {
    __shared__ double sh[64];
    grouped_for<VecG, true>(tab, stride, npatch, [&](const VecG& g, int item) { vec_body<double, OP>(g.a, g.sc, g.part, item, g.nblk, sh); });
}

template <int OP>
__global__ void __launch_bounds__(kRedThreads) k_finish_grouped(const unsigned char* __restrict__ tab, int stride, int npatch) {
    __shared__ double sh[64];
    grouped_for<FinG, true>(tab, stride, npatch, [&](const FinG& g, int) { finish_body<OP>(g.sc, g.part, g.nblk, sh); });
}

constexpr int vec_kind(int op) {
    return op == V_P ? GK_VEC_P : op == V_DOT_RV ? GK_VEC_DOT_RV : op == V_S ? GK_VEC_S : op == V_DOT_TS ? GK_VEC_DOT_TS
         : op == V_XR ? GK_VEC_XR : GK_NONE;
}
constexpr int fin_kind(int op) {
    return op == V_DOT_RV ? GK_FIN_DOT_RV : op == V_S ? GK_FIN_S : op == V_DOT_TS ? GK_FIN_DOT_TS : op == V_XR ? GK_FIN_XR
         : GK_NONE;
}

template <typename T, int OP>
cudaError_t vec(const VArgs<T>& a, const KScal* sc, double* part, cudaStream_t s) {
    const int nblk = red_blocks(a.N);
    if (g_rec) {
        if (sizeof(T) != 8 || vec_kind(OP) == GK_NONE) {
            g_rec->unsupported = true;
            return cudaSuccess;
        }
        VecG g{*reinterpret_cast<const VArgs<double>*>(&a), sc, part, nblk};
        record_launch(vec_kind(OP), g, nblk, kRedThreads, 0, OP == V_DOT_TS ? &sc->skip2 : &sc->skip1);
        return cudaSuccess;
    }
    launch_begin(S_KRYLOV, s);
    k_vec<T, OP><<<nblk, kRedThreads, 0, s>>>(a, sc, part);
    launch_end(S_KRYLOV, s);
    return cudaGetLastError();
}

template <int OP>
cudaError_t fin(KScal* sc, const double* part, size_t N, cudaStream_t s) {
    const int nblk = red_blocks(N);
    if (g_rec) {
        if (fin_kind(OP) == GK_NONE) {
            g_rec->unsupported = true;
            return cudaSuccess;
        }
        FinG g{sc, part, nblk};
        record_launch(fin_kind(OP), g, 1, kRedThreads, 0, OP == V_DOT_TS ? &sc->skip2 : &sc->skip1);
        return cudaSuccess;
    }
    launch_begin(S_KRYLOV, s);
    k_finish<OP><<<1, kRedThreads, 0, s>>>(sc, part, nblk);
    launch_end(S_KRYLOV, s);
    return cudaGetLastError();
}

}  // namespace

#define KTRY(x)                                   \
    do {                                          \
        if ((x) != cudaSuccess) return MFWQ_ECUDA; \
    } while (0)
#define STRY(x)                        \
    do {                               \
        int _st = (x);                 \
        if (_st != MFWQ_OK) return _st; \
    } while (0)

template <typename T>
static VArgs<T> vargs(const KrylovBufs<T>& b, const T* f, T* x, bool x_given, size_t N) {
    VArgs<T> a;
    a.N = N;
    a.f = f;
    a.x = x;
    a.r = b.r;
    a.rhat = b.rhat;
    a.p = b.p;
    a.v = b.v;
    a.s = b.s;
    a.t = b.t;
    a.ph = b.ph;
    a.sh = b.sh;
    a.x_given = x_given ? 1 : 0;
    return a;
}

template <typename T>
int krylov_enqueue_init(const LinOp<T>& A, const T* f, T* x, bool x_given, double rtol, const KrylovBufs<T>& b,
                        KScal* dsc, double* part, size_t N, cudaStream_t s) {
    VArgs<T> a = vargs(b, f, x, x_given, N);
    KScal init{};
    init.rtol = rtol;  // everything else is set by the init finish kernel
    KTRY(cudaMemcpyAsync(dsc, &init, sizeof(KScal), cudaMemcpyHostToDevice, s));
    if (x_given) {
        STRY(A(x, b.v, nullptr));  // r = f - A x0
        STRY(axpby_into(f, b.v, b.r, N, s));
    }
    KTRY((vec<T, V_INIT>(a, dsc, part, s)));
    KTRY(fin<V_INIT>(dsc, part, N, s));
    return MFWQ_OK;
}

template <typename T>
int krylov_enqueue_iter(const LinOp<T>& A, const LinOp<T>& P, const T* f, T* x, const KrylovBufs<T>& b, KScal* dsc,
                        double* part, size_t N, cudaStream_t s) {
    VArgs<T> a = vargs(b, f, x, false, N);
    const int* skip1 = &dsc->skip1;
    const int* skip2 = &dsc->skip2;
    KTRY((vec<T, V_P>(a, dsc, part, s)));
    STRY(P(b.p, b.ph, skip1));
    STRY(A(b.ph, b.v, skip1));
    KTRY((vec<T, V_DOT_RV>(a, dsc, part, s)));
    KTRY(fin<V_DOT_RV>(dsc, part, N, s));
    KTRY((vec<T, V_S>(a, dsc, part, s)));
    KTRY(fin<V_S>(dsc, part, N, s));
    STRY(P(b.s, b.sh, skip2));
    STRY(A(b.sh, b.t, skip2));
    KTRY((vec<T, V_DOT_TS>(a, dsc, part, s)));
    KTRY(fin<V_DOT_TS>(dsc, part, N, s));
    KTRY((vec<T, V_XR>(a, dsc, part, s)));
    KTRY(fin<V_XR>(dsc, part, N, s));
    return MFWQ_OK;
}

void krylov_result(const KScal& h, int* iters, double* relres, int* status) {
    *iters = h.iters;
    *relres = h.f2 > 0 ? std::sqrt(h.r2 / h.f2) : 0.0;
    int st = h.status;
    if (st == MFWQ_OK && !(h.r2 <= h.tol2) && h.f2 > 0) st = MFWQ_ENOCONV;
    *status = st;
}

template <typename T>
int bicgstab(const LinOp<T>& A, const LinOp<T>& P, const T* f, T* x, bool x_given, double rtol, int maxit,
             const KrylovBufs<T>& b, KScal* dsc, KScal* hsc, double* part, size_t N, cudaStream_t s, int check_every,
             double* hist, int* iters, double* relres, int* status, int graph_chunk) {
    STRY(krylov_enqueue_init<T>(A, f, x, x_given, rtol, b, dsc, part, N, s));
    KTRY(cudaMemcpyAsync(hsc, dsc, sizeof(KScal), cudaMemcpyDeviceToHost, s));
    KTRY(cudaStreamSynchronize(s));
    if (hist) hist[0] = hsc->f2 > 0 ? std::sqrt(hsc->r2 / hsc->f2) : 0.0;
    if (!hsc->skip1) {
        if (check_every < 1) check_every = 1;
        // graph_chunk > 1: that many iterations captured once into a CUDA graph, launched
        // between host checks (iterations after convergence are skipped on the device)
        cudaGraphExec_t exec = nullptr;
        if (graph_chunk > 1 && !hist && s != nullptr && maxit >= graph_chunk) {
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                int cst = MFWQ_OK;
                for (int k = 0; k < graph_chunk && cst == MFWQ_OK; ++k)
                    cst = krylov_enqueue_iter<T>(A, P, f, x, b, dsc, part, N, s);
                const cudaError_t ce = cudaStreamEndCapture(s, &graph);
                if (cst != MFWQ_OK || ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
                    exec = nullptr;
                if (graph) cudaGraphDestroy(graph);
            }
            cudaGetLastError();
        }
        int it = 0;
        while (exec && it + graph_chunk <= maxit) {
            if (cudaGraphLaunch(exec, s) != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                return MFWQ_ECUDA;
            }
            it += graph_chunk;
            KTRY(cudaMemcpyAsync(hsc, dsc, sizeof(KScal), cudaMemcpyDeviceToHost, s));
            KTRY(cudaStreamSynchronize(s));
            if (hsc->skip1) break;
        }
        if (exec) cudaGraphExecDestroy(exec);
        for (; it < maxit && !hsc->skip1; ++it) {
            STRY(krylov_enqueue_iter<T>(A, P, f, x, b, dsc, part, N, s));
            if ((it + 1) % check_every == 0 || it + 1 == maxit || hist) {
                KTRY(cudaMemcpyAsync(hsc, dsc, sizeof(KScal), cudaMemcpyDeviceToHost, s));
                KTRY(cudaStreamSynchronize(s));
                if (hist) hist[hsc->iters] = hsc->f2 > 0 ? std::sqrt(hsc->r2 / hsc->f2) : 0.0;
                if (hsc->skip1) break;
            }
        }
    }
    KTRY(cudaMemcpyAsync(hsc, dsc, sizeof(KScal), cudaMemcpyDeviceToHost, s));
    KTRY(cudaStreamSynchronize(s));
    krylov_result(*hsc, iters, relres, status);
    return MFWQ_OK;
}

// ---------------------------------------------------------------- small vector helpers
namespace {
template <typename T>
__global__ void k_axpby_into(const T* __restrict__ f, const T* __restrict__ v, T* __restrict__ r, size_t N) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) r[i] = f[i] - v[i];
}
__global__ void k_norm2(const double* __restrict__ x, size_t N, double* part) {
    __shared__ double sh[64];
    double a = 0.0, b = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) a += x[i] * x[i];
    block_sum2(a, b, sh);
    if (threadIdx.x == 0) part[2 * blockIdx.x] = a, part[2 * blockIdx.x + 1] = 0.0;
}
__global__ void k_sum_parts(const double* __restrict__ part, int nblk, double* out) {
    __shared__ double sh[64];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) a += part[2 * i];
    block_sum2(a, b, sh);
    if (threadIdx.x == 0) *out = a;
}
__global__ void k_to_f32_scaled(const double* __restrict__ x, const double* __restrict__ nrm2, float* __restrict__ y, size_t N) {
    const double inv = 1.0 / sqrt(*nrm2);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
        y[i] = (float)(x[i] * inv);
}
__global__ void k_add_f32_scaled(double* __restrict__ u, const float* __restrict__ d, const double* __restrict__ nrm2, size_t N) {
    const double sc = sqrt(*nrm2);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
        u[i] += sc * (double)d[i];
}
template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ x, D* __restrict__ y, size_t N, const int* skip) {
    if (skip && *skip) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
        y[i] = (D)x[i];
}
}  // namespace

template <typename S, typename D>
int convert_into(const S* x, D* y, size_t N, const int* skip, cudaStream_t s) {
    launch_begin(S_FD_TC, s);
    k_convert<S, D><<<kRedBlocks, kRedThreads, 0, s>>>(x, y, N, skip);
    launch_end(S_FD_TC, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}
template int convert_into<double, float>(const double*, float*, size_t, const int*, cudaStream_t);
template int convert_into<float, double>(const float*, double*, size_t, const int*, cudaStream_t);

template <typename T>
int axpby_into(const T* f, const T* v, T* r, size_t N, cudaStream_t s) {
    launch_begin(S_KRYLOV, s);
    k_axpby_into<T><<<kRedBlocks, kRedThreads, 0, s>>>(f, v, r, N);
    launch_end(S_KRYLOV, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}

int norm2_into(const double* x, size_t N, double* part, double* out, cudaStream_t s) {
    launch_begin(S_KRYLOV, s);
    k_norm2<<<kRedBlocks, kRedThreads, 0, s>>>(x, N, part);
    launch_end(S_KRYLOV, s);
    launch_begin(S_KRYLOV, s);
    k_sum_parts<<<1, kRedThreads, 0, s>>>(part, kRedBlocks, out);
    launch_end(S_KRYLOV, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}

int to_f32_scaled(const double* x, const double* nrm2, float* y, size_t N, cudaStream_t s) {
    launch_begin(S_KRYLOV, s);
    k_to_f32_scaled<<<kRedBlocks, kRedThreads, 0, s>>>(x, nrm2, y, N);
    launch_end(S_KRYLOV, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}

int add_f32_scaled(double* u, const float* d, const double* nrm2, size_t N, cudaStream_t s) {
    launch_begin(S_KRYLOV, s);
    k_add_f32_scaled<<<kRedBlocks, kRedThreads, 0, s>>>(u, d, nrm2, N);
    launch_end(S_KRYLOV, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}

bool grouped_launch_krylov(int kind, const unsigned char* tab, int stride, int npatch, int grid, int smem,
                           cudaStream_t s) {
    (void)smem;
    switch (kind) {
        case GK_VEC_P: k_vec_grouped<V_P><<<grid, kRedThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_VEC_DOT_RV: k_vec_grouped<V_DOT_RV><<<grid, kRedThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_VEC_S: k_vec_grouped<V_S><<<grid, kRedThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_VEC_DOT_TS: k_vec_grouped<V_DOT_TS><<<grid, kRedThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_VEC_XR: k_vec_grouped<V_XR><<<grid, kRedThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_FIN_DOT_RV: k_finish_grouped<V_DOT_RV><<<grid, kRedThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_FIN_S: k_finish_grouped<V_S><<<grid, kRedThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_FIN_DOT_TS: k_finish_grouped<V_DOT_TS><<<grid, kRedThreads, 0, s>>>(tab, stride, npatch); return true;
        case GK_FIN_XR: k_finish_grouped<V_XR><<<grid, kRedThreads, 0, s>>>(tab, stride, npatch); return true;
        default: return false;
    }
}

template int axpby_into<double>(const double*, const double*, double*, size_t, cudaStream_t);
template int axpby_into<float>(const float*, const float*, float*, size_t, cudaStream_t);
template int krylov_enqueue_init<double>(const LinOp<double>&, const double*, double*, bool, double,
                                          const KrylovBufs<double>&, KScal*, double*, size_t, cudaStream_t);
template int krylov_enqueue_init<float>(const LinOp<float>&, const float*, float*, bool, double, const KrylovBufs<float>&,
                                         KScal*, double*, size_t, cudaStream_t);
template int krylov_enqueue_iter<double>(const LinOp<double>&, const LinOp<double>&, const double*, double*,
                                          const KrylovBufs<double>&, KScal*, double*, size_t, cudaStream_t);
template int krylov_enqueue_iter<float>(const LinOp<float>&, const LinOp<float>&, const float*, float*,
                                         const KrylovBufs<float>&, KScal*, double*, size_t, cudaStream_t);
template int bicgstab<double>(const LinOp<double>&, const LinOp<double>&, const double*, double*, bool, double, int,
                              const KrylovBufs<double>&, KScal*, KScal*, double*, size_t, cudaStream_t, int, double*, int*,
                              double*, int*, int);
template int bicgstab<float>(const LinOp<float>&, const LinOp<float>&, const float*, float*, bool, double, int,
                             const KrylovBufs<float>&, KScal*, KScal*, double*, size_t, cudaStream_t, int, double*, int*,
                             double*, int*, int);

}  // namespace mfwq
