// Forward x-stage kernels of the MF-WQ apply (Algorithm 2, Section 3.2) for
// sm_103a: the fused last trial contraction, pointwise coefficient product
// and first test contraction along direction 1, in seven launch shapes the
// autotuner chooses from (mappings 0-3 per (line, item) or per item over the
// block's lines, with or without bulk-copy prefetch; 4-5 two-row tiles; 6 the
// stencil form for translation-invariant interiors), each also with a
// reduced shared-memory carveout (mappings 0-5).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "apply_common.cuh"
#include "grouped.h"
#include "ptx_async.cuh"
#include "stencil_x.cuh"

namespace mfwq {

namespace {

using stx::kSeg;
using stx::kStLines;
using stx::st_load_y;
using stx::st_stride;
using stx::st_test;
using stx::st_trial;
using stx::st_bnd_load;
using stx::st_bnd_count;
using stx::kStBndMax;

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
//  MODE 2, 3: the mappings of MODE 0, 1 with the block's inputs (its three
//          Y slabs and six coefficient slabs, all contiguous) prefetched into
//          shared memory by bulk copies (cp.async.bulk) that complete on one
//          mbarrier, so every HBM read of the block is in flight at once and
//          the coefficient products read shared memory.  Needs LINES *
//          sizeof(T) to be a multiple of 16 and 16-byte aligned slabs.
template <typename T, int LINES>
__device__ bool xstage_prefetch(const XArgs<T>& a, const T* __restrict__ y0, const T* __restrict__ y1,
                                const T* __restrict__ y2, int line0, int nl, T* sY, T* sC, uint64_t* mbar, int* err) {
    const int n1 = a.n1, nq1 = a.nq1;
    if (nl == LINES) {
        const uint32_t mb = ptx::smem_u32(mbar);
        if (threadIdx.x == 0) {
            ptx::mbar_init(mb, 1);
            ptx::fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t yb = (uint32_t)(LINES * n1 * sizeof(T)), cb = (uint32_t)(LINES * nq1 * sizeof(T));
            ptx::mbar_expect_tx(mb, 3 * yb + 6 * cb);
            const size_t yo = (size_t)line0 * n1, co = (size_t)line0 * nq1;
            ptx::bulk_g2s(ptx::smem_u32(sY), y0 + yo, yb, mb);
            ptx::bulk_g2s(ptx::smem_u32(sY + LINES * n1), y1 + yo, yb, mb);
            ptx::bulk_g2s(ptx::smem_u32(sY + 2 * LINES * n1), y2 + yo, yb, mb);
            for (int s = 0; s < 6; ++s) ptx::bulk_g2s(ptx::smem_u32(sC + s * LINES * nq1), a.C + s * a.cs + co, cb, mb);
        }
        const bool ok = ptx::mbar_wait(mb, 0);
        if (__syncthreads_and(ok ? 1 : 0)) return true;
        // timed out: record it, give the copies in flight one more bounded wait, give up on the block
        if (threadIdx.x == 0 && err) atomicExch(err, 1);
        ptx::mbar_wait(mb, 0);
        return false;
    }
    // last, partial block: the slabs are shorter than a multiple of 16 bytes, plain loads
    for (int e = threadIdx.x; e < nl * n1; e += blockDim.x) {
        const int l = e / n1, j = e - l * n1;
        const size_t gi = (size_t)(line0 + l) * n1 + j;
        sY[(0 * LINES + l) * n1 + j] = y0[gi];
        sY[(1 * LINES + l) * n1 + j] = y1[gi];
        sY[(2 * LINES + l) * n1 + j] = y2[gi];
    }
    for (int e = threadIdx.x; e < nl * nq1; e += blockDim.x) {
        const int l = e / nq1, q = e - l * nq1;
        const size_t gi = (size_t)(line0 + l) * nq1 + q;
#pragma unroll
        for (int s = 0; s < 6; ++s) sC[(s * LINES + l) * nq1 + q] = a.C[s * a.cs + gi];
    }
    return true;
}

// CARVE (0 or 1) only makes a separate function: CARVE = 1 copies are given a
// smaller preferred shared-memory carveout, so fewer blocks share an SM and
// the band tables they all read stay in a larger L1.
// One block (virtual index bx) of the x stage; smem_raw: its shared memory.
template <typename T, int LINES, int MODE>
__device__ __forceinline__ void xstage_apply_body(const XArgs<T>& a, const T* __restrict__ y0, const T* __restrict__ y1,
                                                  const T* __restrict__ y2, T* __restrict__ tout, size_t tstride, int* err,
                                                  int bx, unsigned char* smem_raw) {
    constexpr bool PF = MODE >= 2;
    constexpr int MAP = MODE & 1;
    // [mbarrier, 16 B if PF][Y: 3][LINES][n1][H: 3][LINES][nq1][C (PF): 6][LINES][nq1]
    T* sY = reinterpret_cast<T*>(smem_raw + (PF ? 16 : 0));
    T* sH = sY + 3 * LINES * a.n1;
    T* sC = sH + 3 * LINES * a.nq1;
    const int line0 = bx * LINES;
    const int nl = min(LINES, a.nlines - line0);
    const int n1 = a.n1, nq1 = a.nq1;
    const int hs = LINES * nq1;
    if (PF) {
        if (!xstage_prefetch<T, LINES>(a, y0, y1, y2, line0, nl, sY, sC, reinterpret_cast<uint64_t*>(smem_raw), err))
            return;
    } else {
        for (int e = threadIdx.x; e < nl * n1; e += blockDim.x) {
            const int l = e / n1, j = e - l * n1;
            const size_t gi = (size_t)(line0 + l) * n1 + j;
            sY[(0 * LINES + l) * n1 + j] = y0[gi];
            sY[(1 * LINES + l) * n1 + j] = y1[gi];
            sY[(2 * LINES + l) * n1 + j] = y2[gi];
        }
    }
    // coefficient field s at (line l, point q): shared-memory slab or HBM
    auto cval = [&](int s, int l, int q) -> T {
        if (PF) return sC[(s * LINES + l) * nq1 + q];
        return a.C[(size_t)s * a.cs + (size_t)(line0 + l) * nq1 + q];
    };
    for (int b = 0; b < 3; ++b) {
        __syncthreads();
        const int bfam = b == 0 ? 1 : 0;
        // symmetric-storage slots of C_(alpha,beta), alpha = 1..3: alpha if alpha = beta, else 2 + alpha + beta
        const int c0 = b == 0 ? 0 : 2 + b;
        const int c1 = b == 1 ? 1 : 3 + b;
        const int c2 = b == 2 ? 2 : 4 + b;
        if (MAP == 0) {
            // points in parity order (even q, then odd q): interior points of one
            // parity have bands of one length, so a warp's lanes leave the tap loop together
            const int half = (nq1 + 1) >> 1;
            for (int e = threadIdx.x; e < nl * nq1; e += blockDim.x) {
                const int l = e / nq1, r = e - l * nq1;
                const int q = r < half ? 2 * r : 2 * (r - half) + 1;
                const int s = a.B.start[q], L = a.B.len[q];
                // the three coefficients are loaded before the tap loop, so their
                // latency overlaps it
                const T k0 = cval(c0, l, q), k1 = cval(c1, l, q), k2 = cval(c2, l, q);
                const T* Y = sY + (b * LINES + l) * n1 + s;
                T g = 0;
                for (int t = 0; t < L; ++t) g = fmaT(a.B.lane(bfam, q, t), Y[t], g);
                T* H = sH + l * nq1 + q;
                H[0 * hs] = k0 * g;
                H[1 * hs] = k1 * g;
                H[2 * hs] = k2 * g;
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
                    T* H = sH + l * nq1 + q;
                    H[0 * hs] = cval(c0, l, q) * g[l];
                    H[1 * hs] = cval(c1, l, q) * g[l];
                    H[2 * hs] = cval(c2, l, q) * g[l];
                }
            }
        }
        __syncthreads();
        // outputs; x-family (a1, b1) = ([alpha = 1], [beta = 1])
        if (MAP == 0) {
            // items (alpha, line, i): first the rows of uniform band length (wnb <= i <
            // n1 - wnb) of all (alpha, line), then the 2 wnb end rows of each, so that
            // the warps walking the longer end bands are few and hold nothing else
            const int nb = a.wnb, ni = n1 - 2 * nb, rows = 3 * nl;
            for (int e = threadIdx.x; e < rows * n1; e += blockDim.x) {
                int row, i;
                if (e < rows * ni) {
                    row = e / ni;
                    i = nb + (e - row * ni);
                } else {
                    const int k = e - rows * ni;
                    row = k / (2 * nb);
                    const int j = k - row * 2 * nb;
                    i = j < nb ? j : ni + j;
                }
                const int al = row / nl, l = row - al * nl;
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

template <typename T, int LINES, int MODE, int CARVE>
__global__ void __launch_bounds__(kThreads) k_xstage_apply(XArgs<T> a, const T* __restrict__ y0, const T* __restrict__ y1,
                                                           const T* __restrict__ y2, T* __restrict__ tout, size_t tstride,
                                                           const int* skip, int* err) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    xstage_apply_body<T, LINES, MODE>(a, y0, y1, y2, tout, tstride, err, blockIdx.x, smem_raw);
}

// Grouped form (batched FP64 solve): mapping 0, 4 lines per block, every patch.
struct XstageG {
    XArgs<double> a;
    const double* y0;
    const double* y1;
    const double* y2;
    double* tout;
    size_t tstride;
    int* err;
};

__global__ void __launch_bounds__(kThreads) k_xstage_grouped(const unsigned char* __restrict__ tab, int stride, int npatch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    grouped_for<XstageG, true>(tab, stride, npatch, [&](const XstageG& p, int item) {
        xstage_apply_body<double, 4, 0>(p.a, p.y0, p.y1, p.y2, p.tout, p.tstride, p.err, item, smem_raw);
    });
}

template <typename T, int MODE, int CARVE>
void launch_xstage(int L, dim3 grid, size_t sm, cudaStream_t st, const XArgs<T>& a, const T* y0, const T* y1, const T* y2,
                   T* tout, size_t tstride, const int* skip, int* err) {
    if (L == 2) k_xstage_apply<T, 2, MODE, CARVE><<<grid, kThreads, sm, st>>>(a, y0, y1, y2, tout, tstride, skip, err);
    else if (L == 8) k_xstage_apply<T, 8, MODE, CARVE><<<grid, kThreads, sm, st>>>(a, y0, y1, y2, tout, tstride, skip, err);
    else k_xstage_apply<T, 4, MODE, CARVE><<<grid, kThreads, sm, st>>>(a, y0, y1, y2, tout, tstride, skip, err);
}

// ---- tiled forward x stage (modes 4 and 5)
// A block owns kTileLines = 8 lines; shared memory holds them lines-innermost
// ([row][8 lines], 16 bytes of padding after every 128 bytes so that lanes a
// few rows apart hit different banks).  A thread owns a tile of two rows of
// B or W (two points, or two outputs) and LG = 4 (mode 4) or 8 (mode 5) lines
// and walks the tile's union window once: per window offset one paired load
// of the two rows' band values and LG-wide vector loads of the lines, 2 * LG
// multiply-adds (4 * LG for the alpha = 2, 3 pair of outputs, which share the
// W family).  Register tiles over rows and lines cut the shared-memory and L1
// traffic per multiply-add several times below one thread per (line, item).
constexpr int kTileLines = 8;

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

// element offset of row r in a lines-innermost slab
template <typename T>
__host__ __device__ __forceinline__ int trow(int r) {
    constexpr int PR = 128 / (kTileLines * (int)sizeof(T));  // rows per 128 bytes: 4 (FP32), 2 (FP64)
    return r * kTileLines + (r / PR) * (16 / (int)sizeof(T));
}

// LG consecutive line values of a lines-innermost row, 16-byte vector loads
template <typename T, int LG>
__device__ __forceinline__ void load_lines(const T* p, T* v) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < LG / 4; ++k) {
            const float4 x = reinterpret_cast<const float4*>(p)[k];
            v[4 * k] = x.x;
            v[4 * k + 1] = x.y;
            v[4 * k + 2] = x.z;
            v[4 * k + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < LG / 2; ++k) {
            const double2 x = reinterpret_cast<const double2*>(p)[k];
            v[2 * k] = x.x;
            v[2 * k + 1] = x.y;
        }
    }
}

template <typename T, int LG>
__device__ __forceinline__ void store_lines(T* p, const T* v) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int k = 0; k < LG / 4; ++k)
            reinterpret_cast<float4*>(p)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < LG / 2; ++k) reinterpret_cast<double2*>(p)[k] = make_double2(v[2 * k], v[2 * k + 1]);
    }
}

template <typename T, int LG, int CARVE>
__global__ void __launch_bounds__(kThreads) k_xstage_tiled(XArgs<T> a, const T* __restrict__ y0, const T* __restrict__ y1,
                                                           const T* __restrict__ y2, T* __restrict__ tout, size_t tstride,
                                                           const int* skip) {
    using T2 = typename Vec2<T>::type;
    constexpr int NG = kTileLines / LG;  // line groups per block
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = a.n1, nq1 = a.nq1;
    const int ysz = trow<T>(n1 + 4), hsz = trow<T>(nq1 + 4);  // slab sizes (whole 128-byte groups)
    T* sY = reinterpret_cast<T*>(smem_raw);  // [3 beta][ysz]: Y rows j
    T* sH = sY + 3 * ysz;                    // [3 alpha][hsz]: H rows q
    const int line0 = blockIdx.x * kTileLines;
    const int nl = min(kTileLines, a.nlines - line0);
    for (int e = threadIdx.x; e < 3 * kTileLines * n1; e += blockDim.x) {
        const int b = e / (kTileLines * n1), rem = e - b * kTileLines * n1;
        const int l = rem / n1, j = rem - l * n1;
        const T* yb = b == 0 ? y0 : (b == 1 ? y1 : y2);
        sY[b * ysz + trow<T>(j) + l] = l < nl ? yb[(size_t)(line0 + l) * n1 + j] : T(0);
    }
    const int ntb = a.BX.ntile, ntw = a.WX.ntile;
    for (int b = 0; b < 3; ++b) {
        __syncthreads();
        const int bfam = b == 0 ? 1 : 0;
        const int cs[3] = {b == 0 ? 0 : 2 + b, b == 1 ? 1 : 3 + b, b == 2 ? 2 : 4 + b};
        // trial: G_b at points 2k, 2k+1 for LG lines, then H^(alpha b) = C_(alpha b) G_b
        for (int it = threadIdx.x; it < ntb * NG; it += blockDim.x) {
            const int g = it / ntb, k = it - g * ntb;
            const int j0 = a.BX.start[k], wl = a.BX.len[k];
            T acc0[LG], acc1[LG];
#pragma unroll
            for (int l = 0; l < LG; ++l) acc0[l] = acc1[l] = 0;
            const T* ys = sY + b * ysz + g * LG;
            for (int u = 0; u < wl; ++u) {
                const T2 bb = *reinterpret_cast<const T2*>(a.BX.pair(bfam, u, k));
                T y[LG];
                load_lines<T, LG>(ys + trow<T>(j0 + u), y);
#pragma unroll
                for (int l = 0; l < LG; ++l) {
                    acc0[l] = fmaT(bb.x, y[l], acc0[l]);
                    acc1[l] = fmaT(bb.y, y[l], acc1[l]);
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int q = 2 * k + r;
                if (q >= nq1) break;
#pragma unroll
                for (int al = 0; al < 3; ++al) {
                    T h[LG];
#pragma unroll
                    for (int l = 0; l < LG; ++l) {
                        const int line = g * LG + l;
                        const T c = line < nl ? a.C[(size_t)cs[al] * a.cs + (size_t)(line0 + line) * nq1 + q] : T(0);
                        h[l] = c * (r == 0 ? acc0[l] : acc1[l]);
                    }
                    store_lines<T, LG>(sH + al * hsz + trow<T>(q) + g * LG, h);
                }
            }
        }
        __syncthreads();
        // test: the alpha = 2, 3 outputs (W family bfam, shared) and the alpha = 1 outputs (family 2 + bfam)
        const int np = ntw * NG;
        for (int it = threadIdx.x; it < 2 * np; it += blockDim.x) {
            const bool two = it < np;
            const int jt = two ? it : it - np;
            const int g = jt / ntw, k = jt - g * ntw;
            const int q0 = a.WX.start[k], wl = a.WX.len[k];
            const int fam = two ? bfam : 2 + bfam;
            const int i0 = 2 * k;
            if (two) {
                T a20[LG], a21[LG], a30[LG], a31[LG];
#pragma unroll
                for (int l = 0; l < LG; ++l) a20[l] = a21[l] = a30[l] = a31[l] = 0;
                const T* h2 = sH + 1 * hsz + g * LG;
                const T* h3 = sH + 2 * hsz + g * LG;
                for (int u = 0; u < wl; ++u) {
                    const T2 w = *reinterpret_cast<const T2*>(a.WX.pair(fam, u, k));
                    T x2[LG], x3[LG];
                    load_lines<T, LG>(h2 + trow<T>(q0 + u), x2);
                    load_lines<T, LG>(h3 + trow<T>(q0 + u), x3);
#pragma unroll
                    for (int l = 0; l < LG; ++l) {
                        a20[l] = fmaT(w.x, x2[l], a20[l]);
                        a21[l] = fmaT(w.y, x2[l], a21[l]);
                        a30[l] = fmaT(w.x, x3[l], a30[l]);
                        a31[l] = fmaT(w.y, x3[l], a31[l]);
                    }
                }
                T* o2 = tout + (size_t)(3 + b) * tstride;
                T* o3 = tout + (size_t)(6 + b) * tstride;
#pragma unroll
                for (int l = 0; l < LG; ++l) {
                    const int line = g * LG + l;
                    if (line >= nl) break;
                    const size_t ob = (size_t)(line0 + line) * n1 + i0;
                    o2[ob] = a20[l];
                    o3[ob] = a30[l];
                    if (i0 + 1 < n1) {
                        o2[ob + 1] = a21[l];
                        o3[ob + 1] = a31[l];
                    }
                }
            } else {
                T a10[LG], a11[LG];
#pragma unroll
                for (int l = 0; l < LG; ++l) a10[l] = a11[l] = 0;
                const T* h1 = sH + g * LG;
                for (int u = 0; u < wl; ++u) {
                    const T2 w = *reinterpret_cast<const T2*>(a.WX.pair(fam, u, k));
                    T x1[LG];
                    load_lines<T, LG>(h1 + trow<T>(q0 + u), x1);
#pragma unroll
                    for (int l = 0; l < LG; ++l) {
                        a10[l] = fmaT(w.x, x1[l], a10[l]);
                        a11[l] = fmaT(w.y, x1[l], a11[l]);
                    }
                }
                T* o1 = tout + (size_t)b * tstride;
#pragma unroll
                for (int l = 0; l < LG; ++l) {
                    const int line = g * LG + l;
                    if (line >= nl) break;
                    const size_t ob = (size_t)(line0 + line) * n1 + i0;
                    o1[ob] = a10[l];
                    if (i0 + 1 < n1) o1[ob + 1] = a11[l];
                }
            }
        }
    }
}

// ---- stencil forward x stage (mode 6): translation-invariant interiors
// Staged outputs of one beta to T^(alpha beta): warp w copies rows w, w + 8, w + 16.
template <typename T, int BETA>
__device__ __forceinline__ void st_copy_out(int n1, int line0, int nl, const T* sT, T* __restrict__ tout,
                                            size_t tstride) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rT = st_stride(n1);
    for (int row = warp; row < 3 * kStLines; row += kStLines) {
        const int al = row >> 3, ll = row & 7;  // kStLines = 8
        if (ll >= nl) continue;
        T* o = tout + (size_t)(3 * al + BETA) * tstride + (size_t)(line0 + ll) * n1;
        const T* src = sT + row * rT;
        for (int i = lane; i < n1; i += 32) o[i] = src[i];
    }
}

// One block = 8 lines.  Per beta two barriers: (trial of beta, copy-out of
// beta - 1) | (test of beta, Y of beta + 1 arriving by cp.async).
template <typename T, int P>
__global__ void __launch_bounds__(kThreads) k_xstage_stencil(XArgs<T> a, StencilD<T> st, const T* __restrict__ y0,
                                                             const T* __restrict__ y1, const T* __restrict__ y2,
                                                             T* __restrict__ tout, size_t tstride, int bnd,
                                                             const int* skip) {
    if (skip && *skip) return;
    const int line0 = blockIdx.x * kStLines;
    const int nl = min(kStLines, a.nlines - line0);
    const int n1 = a.n1;
    if (threadIdx.x < 9) {  // the block's inputs (6 coefficient rows, 3 Y slabs) requested into L2 up front
        const int f = threadIdx.x;
        if (f < 6)
            ptx::prefetch_l2_range(a.C + (size_t)f * a.cs + (size_t)line0 * a.nq1, sizeof(T) * (size_t)nl * a.nq1);
        else
            ptx::prefetch_l2_range((f == 6 ? y0 : f == 7 ? y1 : y2) + (size_t)line0 * n1, sizeof(T) * (size_t)nl * n1);
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sY = reinterpret_cast<T*>(smem_raw);             // [8][rY]: Y rows of one beta
    T* sT = sY + kStLines * st_stride(n1);              // [3 alpha][8][rT]: staged outputs of one beta
    T* sH = sT + 3 * kStLines * st_stride(n1);          // [3 alpha][8][rG]
    const int rY = st_stride(n1), rT = st_stride(n1), rG = st_stride(a.nq1);
    // boundary weights of the test side, staged once for the block's three betas
    T* sW = bnd ? sH + 3 * kStLines * rG : nullptr;
    if (bnd) st_bnd_load<T, P>(a, st, sW);
    st_load_y(y0, n1, line0, nl, sY, rY);
    ptx::cp_async_commit();
    ptx::cp_async_wait_all();
    __syncthreads();
    st_trial<T, P, 0>(a, st, line0, nl, sY, sH, rY, rG);
    __syncthreads();
    st_load_y(y1, n1, line0, nl, sY, rY);
    ptx::cp_async_commit();
    st_test<T, P, 0>(a, st, sH, sT, rG, rT, sW);
    ptx::cp_async_wait_all();
    __syncthreads();
    st_copy_out<T, 0>(n1, line0, nl, sT, tout, tstride);
    st_trial<T, P, 1>(a, st, line0, nl, sY, sH, rY, rG);
    __syncthreads();
    st_load_y(y2, n1, line0, nl, sY, rY);
    ptx::cp_async_commit();
    st_test<T, P, 1>(a, st, sH, sT, rG, rT, sW);
    ptx::cp_async_wait_all();
    __syncthreads();
    st_copy_out<T, 1>(n1, line0, nl, sT, tout, tstride);
    st_trial<T, P, 2>(a, st, line0, nl, sY, sH, rY, rG);
    __syncthreads();
    st_test<T, P, 2>(a, st, sH, sT, rG, rT, sW);
    __syncthreads();
    st_copy_out<T, 2>(n1, line0, nl, sT, tout, tstride);
}

constexpr size_t kStencilSmemCap = 227 * 1024;  // opt-in shared memory per block

// Shared memory for the staged boundary weights of the stencil test side
// (st_bnd_load), 0 when there are more than kStBndMax boundary outputs.
template <typename T>
size_t stencil_bnd_bytes(const StencilD<T>& S, int n1) {
    const int nb = st_bnd_count(S.i_lo, S.i_hi, n1);
    if (nb > kStBndMax) return 0;
    return (size_t)4 * nb * (3 * S.P + 1) * sizeof(T) + (size_t)2 * nb * sizeof(int);
}

// The same x stage with the coefficient evaluated in the block (CoeffField):
// kappa of the block's 8 lines into shared memory first, then the three betas
// with C = kappa G; nothing of C is read from HBM.
template <int P>
__global__ void __launch_bounds__(kThreads) k_xstage_stencil_otf(XArgs<float> a, StencilD<float> st, CoeffField cf,
                                                                 const float* __restrict__ y0,
                                                                 const float* __restrict__ y1,
                                                                 const float* __restrict__ y2, float* __restrict__ tout,
                                                                 size_t tstride, int nq2, const int* skip) {
    if (skip && *skip) return;
    const int line0 = blockIdx.x * kStLines;
    const int nl = min(kStLines, a.nlines - line0);
    const int n1 = a.n1;
    if (threadIdx.x < 3) {
        const int f = threadIdx.x;
        ptx::prefetch_l2_range((f == 0 ? y0 : f == 1 ? y1 : y2) + (size_t)line0 * n1, sizeof(float) * (size_t)nl * n1);
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sY = reinterpret_cast<float*>(smem_raw);
    const int rY = st_stride(n1), rT = st_stride(n1), rG = st_stride(a.nq1);
    float* sT = sY + kStLines * rY;
    float* sH = sT + 3 * kStLines * rT;
    float* sK = sH + 3 * kStLines * rG;      // [8][rG]: kappa of the block's lines
    float* sAB = sK + kStLines * rG;         // [8][kMaxModes][4]
    st_load_y(y0, n1, line0, nl, sY, rY);
    ptx::cp_async_commit();
    stx::st_kappa(cf, line0, nl, a.nq1, nq2, sK, rG, sAB);
    ptx::cp_async_wait_all();
    __syncthreads();
    stx::st_trial_otf<P, 0>(a, st, nl, sY, sH, rY, rG, sK, rG, cf.g6);
    __syncthreads();
    st_load_y(y1, n1, line0, nl, sY, rY);
    ptx::cp_async_commit();
    st_test<float, P, 0>(a, st, sH, sT, rG, rT);
    ptx::cp_async_wait_all();
    __syncthreads();
    st_copy_out<float, 0>(n1, line0, nl, sT, tout, tstride);
    stx::st_trial_otf<P, 1>(a, st, nl, sY, sH, rY, rG, sK, rG, cf.g6);
    __syncthreads();
    st_load_y(y2, n1, line0, nl, sY, rY);
    ptx::cp_async_commit();
    st_test<float, P, 1>(a, st, sH, sT, rG, rT);
    ptx::cp_async_wait_all();
    __syncthreads();
    st_copy_out<float, 1>(n1, line0, nl, sT, tout, tstride);
    stx::st_trial_otf<P, 2>(a, st, nl, sY, sH, rY, rG, sK, rG, cf.g6);
    __syncthreads();
    st_test<float, P, 2>(a, st, sH, sT, rG, rT);
    __syncthreads();
    st_copy_out<float, 2>(n1, line0, nl, sT, tout, tstride);
}

}  // namespace

int xstage_otf_smem_bytes(int n1, int nq1) {
    return (int)(((size_t)kStLines * (4 * (size_t)st_stride(n1) + 4 * (size_t)st_stride(nq1)) +
                  (size_t)kStLines * kMaxModes * 4) * sizeof(float));
}

static void launch_stencil_otf(const StencilD<float>& S, const CoeffField& cf, int nlines, int nq2, size_t sm,
                               cudaStream_t st, const XArgs<float>& a, const float* y0, const float* y1,
                               const float* y2, float* tout, size_t tstride, const int* skip) {
    const dim3 grid((nlines + kStLines - 1) / kStLines);
    switch (S.P) {
        case 2: k_xstage_stencil_otf<2><<<grid, kThreads, sm, st>>>(a, S, cf, y0, y1, y2, tout, tstride, nq2, skip); break;
        case 3: k_xstage_stencil_otf<3><<<grid, kThreads, sm, st>>>(a, S, cf, y0, y1, y2, tout, tstride, nq2, skip); break;
        case 4: k_xstage_stencil_otf<4><<<grid, kThreads, sm, st>>>(a, S, cf, y0, y1, y2, tout, tstride, nq2, skip); break;
        case 5: k_xstage_stencil_otf<5><<<grid, kThreads, sm, st>>>(a, S, cf, y0, y1, y2, tout, tstride, nq2, skip); break;
        case 6: k_xstage_stencil_otf<6><<<grid, kThreads, sm, st>>>(a, S, cf, y0, y1, y2, tout, tstride, nq2, skip); break;
        case 7: k_xstage_stencil_otf<7><<<grid, kThreads, sm, st>>>(a, S, cf, y0, y1, y2, tout, tstride, nq2, skip); break;
        case 8: k_xstage_stencil_otf<8><<<grid, kThreads, sm, st>>>(a, S, cf, y0, y1, y2, tout, tstride, nq2, skip); break;
        default: break;  // unreachable: the field path needs the stencil tables (P <= kStencilMaxP), checked when set
    }
}

int configure_xstage_otf_smem(int bytes) {
    cudaError_t e = cudaSuccess;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    e = cudaFuncSetAttribute(k_xstage_stencil_otf<2>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_stencil_otf<3>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_stencil_otf<4>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_stencil_otf<5>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_stencil_otf<6>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_stencil_otf<7>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_stencil_otf<8>, A, bytes);
    return e == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}

template <typename T>
void launch_stencil(const StencilD<T>& S, int nlines, size_t sm, cudaStream_t st, const XArgs<T>& a, const T* y0,
                    const T* y1, const T* y2, T* tout, size_t tstride, const int* skip) {
    const dim3 grid((nlines + kStLines - 1) / kStLines);
    size_t bb = stencil_bnd_bytes(S, a.n1);
    if (sm + bb > kStencilSmemCap) bb = 0;  // the configured limit (configure_forward_xstage_smem)
    const int bnd = bb > 0 ? 1 : 0;
    sm += bb;
    switch (S.P) {
        case 2: k_xstage_stencil<T, 2><<<grid, kThreads, sm, st>>>(a, S, y0, y1, y2, tout, tstride, bnd, skip); break;
        case 3: k_xstage_stencil<T, 3><<<grid, kThreads, sm, st>>>(a, S, y0, y1, y2, tout, tstride, bnd, skip); break;
        case 4: k_xstage_stencil<T, 4><<<grid, kThreads, sm, st>>>(a, S, y0, y1, y2, tout, tstride, bnd, skip); break;
        case 5: k_xstage_stencil<T, 5><<<grid, kThreads, sm, st>>>(a, S, y0, y1, y2, tout, tstride, bnd, skip); break;
        case 6: k_xstage_stencil<T, 6><<<grid, kThreads, sm, st>>>(a, S, y0, y1, y2, tout, tstride, bnd, skip); break;
        case 7: k_xstage_stencil<T, 7><<<grid, kThreads, sm, st>>>(a, S, y0, y1, y2, tout, tstride, bnd, skip); break;
        case 8: k_xstage_stencil<T, 8><<<grid, kThreads, sm, st>>>(a, S, y0, y1, y2, tout, tstride, bnd, skip); break;
        default: break;  // unreachable: the stencil tables exist only for P <= kStencilMaxP (checked at dispatch)
    }
}

template <typename T, int CARVE>
void launch_xstage_mode(int mode, int L, dim3 grid, size_t sm, cudaStream_t st, const XArgs<T>& a, const T* y0,
                        const T* y1, const T* y2, T* tout, size_t tstride, const int* skip, int* err) {
    if (mode == 4) k_xstage_tiled<T, 4, CARVE><<<grid, kThreads, sm, st>>>(a, y0, y1, y2, tout, tstride, skip);
    else if (mode == 5) k_xstage_tiled<T, 8, CARVE><<<grid, kThreads, sm, st>>>(a, y0, y1, y2, tout, tstride, skip);
    else if (mode == 1) launch_xstage<T, 1, CARVE>(L, grid, sm, st, a, y0, y1, y2, tout, tstride, skip, err);
    else if (mode == 2) launch_xstage<T, 2, CARVE>(L, grid, sm, st, a, y0, y1, y2, tout, tstride, skip, err);
    else if (mode == 3) launch_xstage<T, 3, CARVE>(L, grid, sm, st, a, y0, y1, y2, tout, tstride, skip, err);
    else launch_xstage<T, 0, CARVE>(L, grid, sm, st, a, y0, y1, y2, tout, tstride, skip, err);
}

template <typename T>
cudaError_t launch_forward_xstage(const OpCtx<T>& c, const XArgs<T>& a, const T* y0, const T* y1, const T* y2,
                                  T* tout, size_t tstride, const int* skip) {
    const DirD<T>& d1 = c.d[0];
    const int n1 = d1.n, q1 = d1.nq;
    const int nlines = a.nlines;
    if (g_rec) {  // recorded as mapping 0 with 4 lines per block, the form every patch can share
        if constexpr (sizeof(T) == 8) {
            XstageG p{a, y0, y1, y2, tout, tstride, c.err};
            record_launch(GK_XSTAGE0, p, (nlines + 3) / 4, kThreads, xstage_smem_bytes(8, n1, q1, 4, 0), skip);
        } else {
            g_rec->unsupported = true;
        }
        return cudaSuccess;
    }
        int L = c.xlines == 2 || c.xlines == 8 ? c.xlines : 4;
        int mode = c.xmode >= 0 && c.xmode <= 6 ? c.xmode : 0;
        if (mode >= 4) L = mode == 6 ? kStLines : kTileLines;
        if (!xstage_mode_valid((int)sizeof(T), n1, q1, L, mode) || (mode >= 2 && mode <= 3 && c.cs % 4 != 0) ||
            (mode == 6 && (!d1.SX.ok || d1.SX.P < 2 || d1.SX.P > kStencilMaxP))) {
            mode = 0;
            L = 4;
        }
        if constexpr (sizeof(T) == 4) {
            if (c.cf) {  // coefficient evaluated in the x stage: the stencil form only
                if (!d1.SX.ok || d1.SX.P < 2 || d1.SX.P > kStencilMaxP) return cudaErrorInvalidValue;
                launch_stencil_otf(d1.SX, *c.cf, nlines, c.d[1].nq, (size_t)xstage_otf_smem_bytes(n1, q1), c.stream, a,
                                   y0, y1, y2, tout, tstride, skip);
                return cudaGetLastError();
            }
        }
        const size_t sm = (size_t)xstage_smem_bytes((int)sizeof(T), n1, q1, L, mode);
        dim3 grid((nlines + L - 1) / L);
        if (mode == 6) launch_stencil<T>(d1.SX, nlines, sm, c.stream, a, y0, y1, y2, tout, tstride, skip);
        else if (c.xcarve) launch_xstage_mode<T, 1>(mode, L, grid, sm, c.stream, a, y0, y1, y2, tout, tstride, skip, c.err);
        else launch_xstage_mode<T, 0>(mode, L, grid, sm, c.stream, a, y0, y1, y2, tout, tstride, skip, c.err);
    return cudaGetLastError();
}

int xstage_smem_bytes(int elem_size, int n1, int nq1, int lines, int mode) {
    if (mode == 6)  // stencil: Y rows of 8 lines, staged outputs and H rows of 8 lines x 3 alpha (+ boundary weights)
        return (int)((size_t)kStLines * (4 * (size_t)st_stride(n1) + 3 * (size_t)st_stride(nq1)) * elem_size);
    if (mode >= 4) {  // tiled: two lines-innermost slabs of 3 x (rows + 4) padded rows
        const int pr = 128 / (kTileLines * elem_size), pad = 16 / elem_size;
        auto tr = [&](int r) { return (size_t)r * kTileLines + (size_t)(r / pr) * pad; };
        return (int)(3 * (tr(n1 + 4) + tr(nq1 + 4)) * elem_size);
    }
    size_t e = (size_t)3 * lines * n1 + (size_t)3 * lines * nq1;
    if (mode >= 2) e += (size_t)6 * lines * nq1;
    return (int)(e * elem_size + (mode >= 2 ? 16 : 0));
}

bool xstage_mode_valid(int elem_size, int n1, int nq1, int lines, int mode) {
    if (mode < 0 || mode > 6) return false;
    if (mode == 6 && lines != kStLines) return false;
    if ((mode == 4 || mode == 5) && lines != kTileLines) return false;
    if (mode >= 2 && (lines * elem_size) % 16 != 0) return false;
    return xstage_smem_bytes(elem_size, n1, nq1, lines, mode) <= kXstageSmemMax;
}

constexpr int kReducedCarvePct = 50;  // preferred shared-memory carveout of the CARVE = 1 copies

template <class K>
static cudaError_t set_kernel_smem(K kern, int bytes, int carve) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && carve)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, kReducedCarvePct);
    return e;
}

template <int MODE, int CARVE>
static cudaError_t set_xstage_smem(int bytes) {
    cudaError_t e = set_kernel_smem(k_xstage_apply<double, 2, MODE, CARVE>, bytes, CARVE);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_apply<double, 4, MODE, CARVE>, bytes, CARVE);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_apply<double, 8, MODE, CARVE>, bytes, CARVE);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_apply<float, 2, MODE, CARVE>, bytes, CARVE);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_apply<float, 4, MODE, CARVE>, bytes, CARVE);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_apply<float, 8, MODE, CARVE>, bytes, CARVE);
    return e;
}

template <int CARVE>
static cudaError_t set_xstage_smem_all(int bytes) {
    cudaError_t e = set_xstage_smem<0, CARVE>(bytes);
    if (e == cudaSuccess) e = set_xstage_smem<1, CARVE>(bytes);
    if (e == cudaSuccess) e = set_xstage_smem<2, CARVE>(bytes);
    if (e == cudaSuccess) e = set_xstage_smem<3, CARVE>(bytes);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_tiled<double, 4, CARVE>, bytes, CARVE);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_tiled<double, 8, CARVE>, bytes, CARVE);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_tiled<float, 4, CARVE>, bytes, CARVE);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_tiled<float, 8, CARVE>, bytes, CARVE);
    return e;
}

template <typename T>
static cudaError_t set_stencil_smem(int bytes) {
    cudaError_t e = set_kernel_smem(k_xstage_stencil<T, 2>, bytes, 0);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_stencil<T, 3>, bytes, 0);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_stencil<T, 4>, bytes, 0);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_stencil<T, 5>, bytes, 0);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_stencil<T, 6>, bytes, 0);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_stencil<T, 7>, bytes, 0);
    if (e == cudaSuccess) e = set_kernel_smem(k_xstage_stencil<T, 8>, bytes, 0);
    return e;
}

bool grouped_launch_xstage(int kind, const unsigned char* tab, int stride, int npatch, int grid, int smem,
                           cudaStream_t s) {
    if (kind != GK_XSTAGE0) return false;
    k_xstage_grouped<<<grid, kThreads, smem, s>>>(tab, stride, npatch);
    return true;
}

cudaError_t configure_forward_xstage_smem(int bytes) {
    cudaError_t e = set_xstage_smem_all<0>(bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_xstage_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = set_xstage_smem_all<1>(bytes);
    // the stencil kernels also stage their boundary weights (at most kStBndMax outputs of 3 P + 1 taps, 4 families)
    auto with_bnd = [&](int elem) {
        const size_t b = (size_t)bytes + (size_t)4 * kStBndMax * (3 * kStencilMaxP + 1) * elem + 2 * kStBndMax * 4;
        return (int)std::min<size_t>(b, kStencilSmemCap);
    };
    if (e == cudaSuccess) e = set_stencil_smem<float>(with_bnd(4));
    if (e == cudaSuccess) e = set_stencil_smem<double>(with_bnd(8));
    return e;
}

template cudaError_t launch_forward_xstage<double>(const OpCtx<double>&, const XArgs<double>&, const double*,
                                                  const double*, const double*, double*, size_t, const int*);
template cudaError_t launch_forward_xstage<float>(const OpCtx<float>&, const XArgs<float>&, const float*,
                                                 const float*, const float*, float*, size_t, const int*);

}  // namespace mfwq
