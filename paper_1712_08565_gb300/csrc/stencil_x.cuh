// Device routines of the stencil form of the forward x stage (Algorithm 2,
// Section 3.2, direction 1), shared by the x-stage kernel of the staged apply
// (xstage_kernels.cu) and the fused FP32 apply (fused_apply.cu).  Internal.
//
// Shared-memory rows are addressed through strides the caller chooses: the
// (line, alpha) lanes of the test read 24 rows at one column offset, so any
// odd row stride keeps them on 24 distinct banks.
#pragma once

#include <cuda_runtime.h>

#include "apply_common.cuh"
#include "ptx_async.cuh"

namespace mfwq {
namespace stx {

// For uniform knots the interior rows of B (pairs of points) and W (outputs)
// are one filter shifted along the line (StencilD); boundary rows use the
// band tables.  A block owns 8 lines and takes the three trial gradients
// beta in turn; the block's inputs are requested into L2 when it starts.
//  trial: warp w = line w, lanes = consecutive pairs of points; the pair's
//    window of P + 2 Y values gives G_b at both points (filter taps are kernel
//    parameters), then the three H^(alpha b) = C_(alpha b) G_b with coalesced
//    coefficient loads, stored to shared memory;
//  test: lanes = (line, alpha), 24 of 32; a lane walks segments of 8 outputs
//    of its own row with the window (2P + 15 values) in registers: 8(2P + 1)
//    multiply-adds per window.  Row strides are 1 mod 32 and the alpha slabs
//    8 rows apart, so the 24 lanes hit 24 different banks;
//  outputs staged in shared memory and written out coalesced while the next
//    beta's trial runs; the next beta's Y slab arrives by cp.async during the
//    test, so each beta costs two barriers.
constexpr int kStLines = 8;  // the (line, alpha) lane map and the copy-out assume 8
constexpr int kSeg = 8;
static_assert(kStLines == 8, "stencil x stage: 3 x 8 (line, alpha) lanes per warp");
static_assert(kThreads / 32 == kStLines, "stencil x stage: one warp per line in the trial");

// Longest boundary band rows of degree P (B: the P + 1 basis functions
// nonzero at a point; W: the points in a function's support, at most 3P + 1
// for the WQ rules here).  The boundary loops are unrolled to these lengths,
// taps beyond the row's own length predicated off, and any longer row ends in
// a plain loop; the taps are summed in ascending order either way.
template <int P>
constexpr int kBndB = P + 1;
template <int P>
constexpr int kBndW = 3 * P + 1;

// row stride >= n with stride = 1 (mod 32)
__host__ __device__ inline int st_stride(int n) { return ((n + 30) / 32) * 32 + 1; }

template <typename T, int P, int BF>
__device__ __forceinline__ void st_pair(const StencilD<T>& st, const T* Y, T& g0, T& g1) {
    constexpr int NB = P + 2;
    T a = 0, b = 0;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const T y = Y[t];
        a = fmaT(st.bf[BF][0][t], y, a);
        b = fmaT(st.bf[BF][1][t], y, b);
    }
    g0 = a;
    g1 = b;
}

// Two pairs at once (windows YA and YB), their four FMA chains interleaved;
// each value is summed in the order of st_pair.
template <typename T, int P, int BF>
__device__ __forceinline__ void st_pair2(const StencilD<T>& st, const T* YA, const T* YB, T& a0, T& a1, T& b0, T& b1) {
    constexpr int NB = P + 2;
    T x0 = 0, x1 = 0, z0 = 0, z1 = 0;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const T ya = YA[t], yb = YB[t];
        x0 = fmaT(st.bf[BF][0][t], ya, x0);
        x1 = fmaT(st.bf[BF][1][t], ya, x1);
        z0 = fmaT(st.bf[BF][0][t], yb, z0);
        z1 = fmaT(st.bf[BF][1][t], yb, z1);
    }
    a0 = x0;
    a1 = x1;
    b0 = z0;
    b1 = z1;
}

template <typename T, int P>
__device__ __forceinline__ void st_seg(const T* w, const T* H, T* To) {
    constexpr int NW = 2 * P + 1, WIN = 2 * (kSeg - 1) + NW;
    T h[WIN];
#pragma unroll
    for (int u = 0; u < WIN; ++u) h[u] = H[u];
#pragma unroll
    for (int r = 0; r < kSeg; ++r) {
        T acc = 0;
#pragma unroll
        for (int t = 0; t < NW; ++t) acc = fmaT(w[t], h[2 * r + t], acc);
        To[r] = acc;
    }
}

// FP32: two segments of one row at once, segments A (window at H) and B
// (window at H + 2 kSeg), paired in the packed FP32 FMA (two FMAs per
// instruction, each rounded as by fmaf).  The window is streamed point by
// point; output r takes its taps in ascending order, as in st_seg, so the
// results are bitwise those of two st_seg calls.
template <int P>
__device__ __forceinline__ void st_seg2(const float2* w2, const float* H, float* To) {
    constexpr int NW = 2 * P + 1, WIN = 2 * (kSeg - 1) + NW;
    float2 acc[kSeg];
#pragma unroll
    for (int r = 0; r < kSeg; ++r) acc[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < WIN; ++u) {
        const float2 hh = make_float2(H[u], H[u + 2 * kSeg]);
#pragma unroll
        for (int r = 0; r < kSeg; ++r) {
            const int t = u - 2 * r;
            if (t >= 0 && t < NW) acc[r] = __ffma2_rn(w2[t], hh, acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < kSeg; ++r) {
        To[r] = acc[r].x;
        To[kSeg + r] = acc[r].y;
    }
}

// The Y slab of one beta for this block's lines: warp w copies line w's row
// asynchronously (cp.async) into sY.
template <typename T>
__device__ __forceinline__ void st_load_y(const T* __restrict__ yb, int n1, int line0, int nl, T* sY, int rY) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp >= nl) return;
    const T* src = yb + (size_t)(line0 + warp) * n1;
    T* dst = sY + warp * rY;
    for (int j = lane; j < n1; j += 32) ptx::cp_async_elem(dst + j, src + j);
}

// Trial side of one beta: G_beta at every point of line w (warp w) from its Y
// row, times the three coefficients C_(alpha beta), into the H rows.
template <typename T, int P, int BETA>
__device__ __forceinline__ void st_trial(const XArgs<T>& a, const StencilD<T>& st, int line0, int nl, const T* sY,
                                         T* sH, int rY, int rG) {
    constexpr int BF = BETA == 0 ? 1 : 0;  // trial family: derivative in direction 1 for beta = 1
    const int nq1 = a.nq1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = BETA == 0 ? 0 : 2 + BETA, c1 = BETA == 1 ? 1 : 3 + BETA, c2 = BETA == 2 ? 2 : 4 + BETA;
    if (warp >= nl) return;
    const size_t lb = (size_t)(line0 + warp) * nq1;
    const T* C0 = a.C + (size_t)c0 * a.cs + lb;
    const T* C1 = a.C + (size_t)c1 * a.cs + lb;
    const T* C2 = a.C + (size_t)c2 * a.cs + lb;
    // boundary points of this line: their coefficients (first 32 points) are
    // requested before the interior loop so that the latency overlaps it
    const int nbq = st.q_lo + (nq1 - st.q_hi);
    const int qb = lane < st.q_lo ? lane : st.q_hi + (lane - st.q_lo);
    const bool bl = lane < nbq;
    const T cb0 = bl ? C0[qb] : T(0), cb1 = bl ? C1[qb] : T(0), cb2 = bl ? C2[qb] : T(0);
    // interior pairs: lane = pair k of a chunk of 32; two chunks per pass,
    // the next pass's 12 coefficients loaded before this pass computes
    const int npairs = (st.q_hi - st.q_lo) >> 1;
    const T* Yl = sY + warp * rY + st.jb + lane;
    T* Hl = sH + warp * rG + st.q_lo + 2 * lane;
    const int qo = st.q_lo + 2 * lane;
    auto load6 = [&](int k, T* c) {
        const bool ok = k + lane < npairs;
        const int o = qo + 2 * k;
        c[0] = ok ? C0[o] : T(0);
        c[1] = ok ? C0[o + 1] : T(0);
        c[2] = ok ? C1[o] : T(0);
        c[3] = ok ? C1[o + 1] : T(0);
        c[4] = ok ? C2[o] : T(0);
        c[5] = ok ? C2[o + 1] : T(0);
    };
    T cn[2][6];
    load6(0, cn[0]);
    load6(32, cn[1]);
    for (int k0 = 0; k0 < npairs; k0 += 64) {
        T c[2][6];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 6; ++e) c[h][e] = cn[h][e];
        if (k0 + 64 < npairs) {
            load6(k0 + 64, cn[0]);
            load6(k0 + 96, cn[1]);
        }
        // both pairs of this pass together (the second's window clamped to the
        // first's where it lies beyond the line; its results are not stored)
        if (k0 + lane >= npairs) break;
        const bool okB = k0 + 32 + lane < npairs;
        T g[2][2];
        st_pair2<T, P, BF>(st, Yl + k0, Yl + k0 + (okB ? 32 : 0), g[0][0], g[0][1], g[1][0], g[1][1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !okB) break;
            T* H = Hl + 2 * (k0 + 32 * h);
            H[0] = c[h][0] * g[h][0];
            H[1] = c[h][1] * g[h][1];
            H[kStLines * rG] = c[h][2] * g[h][0];
            H[kStLines * rG + 1] = c[h][3] * g[h][1];
            H[2 * kStLines * rG] = c[h][4] * g[h][0];
            H[2 * kStLines * rG + 1] = c[h][5] * g[h][1];
        }
    }
    // boundary points (band tables)
    for (int k = lane; k < nbq; k += 32) {
        const int q = k < st.q_lo ? k : st.q_hi + (k - st.q_lo);
        const int s0 = a.B.start[q], L = a.B.len[q];
        const T* Y = sY + warp * rY + s0;
        T g = 0;
#pragma unroll
        for (int t = 0; t < kBndB<P>; ++t)
            if (t < L) g = fmaT(a.B.lane(BF, q, t), Y[t], g);
        for (int t = kBndB<P>; t < L; ++t) g = fmaT(a.B.lane(BF, q, t), Y[t], g);
        T* H = sH + warp * rG + q;
        const bool first = k < 32;
        H[0] = (first ? cb0 : C0[q]) * g;
        H[kStLines * rG] = (first ? cb1 : C1[q]) * g;
        H[2 * kStLines * rG] = (first ? cb2 : C2[q]) * g;
    }
}

// kappa(x) = exp(kscale g(x)) at every point of the block's lines line0 ..
// line0 + nl - 1 (global line index q3 * nq2 + q2), into sK[l * rK + q1].  One
// thread per (line, mode) first forms the line's phase coefficients in FP64
// (2A and B, reduced to [-1, 1], each as an unevaluated sum of two floats) in
// sAB [8][kMaxModes][4]; then one thread per point sums the modes in FP32
// with CUDA's sincospif and expf.  The phase 2A s + B is carried as a float
// pair through its reduction modulo 2, and the cosine of the pair is
// cospi(hi) - pi lo sinpi(hi), so the cosine's error is that of sincospif
// (about one FP32 ulp) instead of the rounding of a phase of up to 17
// half-turns.  Ends with a barrier.
__device__ __forceinline__ void st_kappa(const CoeffField& f, int line0, int nl, int nq1, int nq2, float* sK, int rK,
                                         float* sAB) {
    const int nm = f.nmodes;
    if ((int)threadIdx.x < nl * nm) {
        const int l = threadIdx.x / nm, m = threadIdx.x - l * nm;
        const int line = line0 + l, q3 = line / nq2, q2 = line - q3 * nq2;
        const double x2 = f.xq2[q2], x3 = f.xq3[q3];
        double A, C3;
        if (f.geom == MFWQ_GEOM_RING) {
            double sn, cs;
            sincospi(0.5 * x2, &sn, &cs);
            A = f.k[m][0] * cs + f.k[m][1] * sn;
            C3 = f.k[m][2] * x3;
        } else {
            A = f.k[m][0];
            C3 = f.k[m][1] * x2 + f.k[m][2] * x3;
        }
        const double A2 = 2.0 * A;
        double B = 2.0 * C3 + f.phi_pi[m];
        B -= 2.0 * rint(0.5 * B);
        const float hi = (float)A2, bh = (float)B;
        float* o = sAB + (l * kMaxModes + m) * 4;
        o[0] = hi;
        o[1] = (float)(A2 - (double)hi);
        o[2] = bh;
        o[3] = (float)(B - (double)bh);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nl * nq1; e += blockDim.x) {
        const int l = e / nq1, q = e - l * nq1;
        const float sh = f.s1[q], sl = f.s1[nq1 + q];
        const float* ab = sAB + l * kMaxModes * 4;
        float g = 0.f;
        for (int m = 0; m < nm; ++m) {
            const float ah = ab[4 * m], al = ab[4 * m + 1], bh = ab[4 * m + 2], bl = ab[4 * m + 3];
            // phase (ah + al)(sh + sl) + (bh + bl) in half-turns as t + lo, |t| <= 2
            const float p = ah * sh;
            float err = fmaf(ah, sh, -p);  // exact error of the rounded product
            err = fmaf(ah, sl, err);
            err = fmaf(al, sh, err);
            const float n = rintf(0.5f * p);
            const float pr = fmaf(-2.f, n, p);  // p - 2n, exact
            const float t = __fadd_rn(pr, bh);  // TwoSum: t + e = pr + bh exactly
            const float z = __fsub_rn(t, pr);
            const float e = __fadd_rn(__fsub_rn(pr, __fsub_rn(t, z)), __fsub_rn(bh, z));
            const float lo = e + (err + bl);
            // cos(pi (t + lo)) = cospi(t) - pi lo sinpi(t) to first order in lo (|lo| < 1e-6)
            float sn, cs;
            sincospif(t, &sn, &cs);
            g = fmaf(f.a[m], fmaf(-3.14159265f * lo, sn, cs), g);
        }
        sK[l * rK + q] = expf(f.kscale * g);
    }
    __syncthreads();
}

// st_trial with C_(alpha beta)(q) = kappa(q) G_(alpha beta)(q1) (CoeffField):
// kappa of the block's lines from sK, G from the direction-1 table.
template <int P, int BETA>
__device__ __forceinline__ void st_trial_otf(const XArgs<float>& a, const StencilD<float>& st, int nl, const float* sY,
                                             float* sH, int rY, int rG, const float* sK, int rK,
                                             const float* __restrict__ g6) {
    constexpr int BF = BETA == 0 ? 1 : 0;
    const int nq1 = a.nq1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = BETA == 0 ? 0 : 2 + BETA, c1 = BETA == 1 ? 1 : 3 + BETA, c2 = BETA == 2 ? 2 : 4 + BETA;
    if (warp >= nl) return;
    const float* G0 = g6 + (size_t)c0 * nq1;
    const float* G1 = g6 + (size_t)c1 * nq1;
    const float* G2 = g6 + (size_t)c2 * nq1;
    const float* K = sK + warp * rK;
    const int npairs = (st.q_hi - st.q_lo) >> 1;
    const float* Yl = sY + warp * rY + st.jb + lane;
    for (int k = lane; k < npairs; k += 32) {
        const int q = st.q_lo + 2 * k;
        float g0, g1;
        st_pair<float, P, BF>(st, Yl + (k - lane), g0, g1);
        g0 *= K[q];
        g1 *= K[q + 1];
        float* H = sH + warp * rG + q;
        H[0] = __ldg(G0 + q) * g0;
        H[1] = __ldg(G0 + q + 1) * g1;
        H[kStLines * rG] = __ldg(G1 + q) * g0;
        H[kStLines * rG + 1] = __ldg(G1 + q + 1) * g1;
        H[2 * kStLines * rG] = __ldg(G2 + q) * g0;
        H[2 * kStLines * rG + 1] = __ldg(G2 + q + 1) * g1;
    }
    const int nbq = st.q_lo + (nq1 - st.q_hi);
    for (int k = lane; k < nbq; k += 32) {
        const int q = k < st.q_lo ? k : st.q_hi + (k - st.q_lo);
        const int s0 = a.B.start[q], L = a.B.len[q];
        const float* Y = sY + warp * rY + s0;
        float g = 0.f;
#pragma unroll
        for (int t = 0; t < kBndB<P>; ++t)
            if (t < L) g = fmaf(a.B.lane(BF, q, t), Y[t], g);
        for (int t = kBndB<P>; t < L; ++t) g = fmaf(a.B.lane(BF, q, t), Y[t], g);
        g *= K[q];
        float* H = sH + warp * rG + q;
        H[0] = __ldg(G0 + q) * g;
        H[kStLines * rG] = __ldg(G1 + q) * g;
        H[2 * kStLines * rG] = __ldg(G2 + q) * g;
    }
}

// Boundary outputs of the test side (outside the segments of kSeg): the
// interior's leading outputs i < i_lo and those from the last full segment on.
__host__ __device__ inline int st_bnd_count(int i_lo, int i_hi, int n1) {
    const int nseg = (i_hi - i_lo) / kSeg;
    return i_lo + (n1 - (i_lo + nseg * kSeg));
}
constexpr int kStBndMax = 32;  // boundary outputs with their weights staged in shared memory (more: global tables)

// Stages the W bands of the boundary outputs, all four families, zero-padded
// to kBndW<P> taps: sW [4][nb][kBndW<P>], then starts and lengths [2][nb] as ints.
template <typename T, int P>
__device__ __forceinline__ void st_bnd_load(const XArgs<T>& a, const StencilD<T>& st, T* sW) {
    constexpr int KB = kBndW<P>;
    const int n1 = a.n1, nb = st_bnd_count(st.i_lo, st.i_hi, n1);
    const int i_st = n1 - (nb - st.i_lo);
    int* sSL = reinterpret_cast<int*>(sW + 4 * nb * KB);
    for (int e = threadIdx.x; e < 4 * nb * KB; e += blockDim.x) {
        const int f = e / (nb * KB), r = e - f * nb * KB, b = r / KB, t = r - b * KB;
        const int i = b < st.i_lo ? b : i_st + (b - st.i_lo);
        sW[e] = t < a.W.len[i] ? a.W.lane(f, i, t) : T(0);
    }
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int i = b < st.i_lo ? b : i_st + (b - st.i_lo);
        sSL[b] = a.W.start[i];
        sSL[nb + b] = a.W.len[i];
    }
}

// Test side of one beta: the 24 rows (alpha, line) of H against the WQ
// weights of their family, outputs into sT.  sW: the boundary weights staged
// by st_bnd_load (nullptr: read from the band tables).
template <typename T, int P, int BETA>
__device__ __forceinline__ void st_test(const XArgs<T>& a, const StencilD<T>& st, const T* sH, T* sT, int rG, int rT,
                                        const T* sW = nullptr) {
    constexpr int BF = BETA == 0 ? 1 : 0;
    constexpr int NW = 2 * P + 1;
    const int n1 = a.n1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // interior segments of kSeg outputs with the window in registers
    const int nseg = (st.i_hi - st.i_lo) / kSeg;
    const int i_st = st.i_lo + nseg * kSeg;
    const int nbi = st.i_lo + (n1 - i_st);
    if (sizeof(T) == 8) {
        // FP64 is bound by the FP64 pipe, not by shared-memory banks: all 32
        // lanes work, as (line l, segment offset s4) for one alpha per warp pass
        const int l = lane & 7, s4 = lane >> 3;
        const int nm = (nseg + 3) >> 2;
        for (int it = warp; it < 3 * nm; it += kStLines) {
            const int al = it / nm, sg = 4 * (it - al * nm) + s4;
            if (sg >= nseg) continue;
            T w[NW];
#pragma unroll
            for (int t = 0; t < NW; ++t) w[t] = al == 0 ? st.wf[2 + BF][t] : st.wf[BF][t];
            st_seg<T, P>(w, sH + (al * kStLines + l) * rG + st.qw + 2 * kSeg * sg,
                         sT + (al * kStLines + l) * rT + st.i_lo + kSeg * sg);
        }
    } else if (lane < 3 * kStLines) {
        // lane = (line l, alpha al): 24 rows 1 mod 32 apart, conflict-free
        const int al = lane >> 3, l = lane & 7;
        const T* Hl = sH + (al * kStLines + l) * rG + st.qw;
        T* To = sT + (al * kStLines + l) * rT + st.i_lo;
        if constexpr (sizeof(T) == 4) {
            // segment pairs (2m, 2m + 1) in the packed FMA; an odd last segment alone
            float2 w2[NW];
#pragma unroll
            for (int t = 0; t < NW; ++t) {
                const float v = al == 0 ? st.wf[2 + BF][t] : st.wf[BF][t];
                w2[t] = make_float2(v, v);
            }
            const int npr = nseg >> 1;
            for (int sp = warp; sp < npr; sp += kStLines)
                st_seg2<P>(w2, Hl + 4 * kSeg * sp, To + 2 * kSeg * sp);
            if ((nseg & 1) && warp == npr % kStLines) {
                T w[NW];
#pragma unroll
                for (int t = 0; t < NW; ++t) w[t] = w2[t].x;
                st_seg<T, P>(w, Hl + 2 * kSeg * (nseg - 1), To + kSeg * (nseg - 1));
            }
        } else {
            T w[NW];
#pragma unroll
            for (int t = 0; t < NW; ++t) w[t] = al == 0 ? st.wf[2 + BF][t] : st.wf[BF][t];
            for (int sg = warp; sg < nseg; sg += kStLines) st_seg<T, P>(w, Hl + 2 * kSeg * sg, To + kSeg * sg);
        }
    }
    // boundary outputs: one (output, row) item per thread, rows fastest, handed
    // out from the last warp down (the first warps take the extra interior segments)
    for (int it = kThreads - 1 - threadIdx.x; it < nbi * 3 * kStLines; it += kThreads) {
        const int k = it / (3 * kStLines), row = it - k * (3 * kStLines);
        const int i = k < st.i_lo ? k : i_st + (k - st.i_lo);
        const int fam = row < kStLines ? 2 + BF : BF;  // alpha = 1 tests the derivative
        T acc = 0;
        if (sW) {
            const int* sSL = reinterpret_cast<const int*>(sW + 4 * nbi * kBndW<P>);
            const int s0 = sSL[k], L = sSL[nbi + k];
            const T* w = sW + (fam * nbi + k) * kBndW<P>;
            const T* Hr = sH + row * rG + s0;
#pragma unroll
            for (int t = 0; t < kBndW<P>; ++t)
                if (t < L) acc = fmaT(w[t], Hr[t], acc);
        } else {
            const int s0 = a.W.start[i], L = a.W.len[i];
            const T* Hr = sH + row * rG + s0;
#pragma unroll
            for (int t = 0; t < kBndW<P>; ++t)
                if (t < L) acc = fmaT(a.W.lane(fam, i, t), Hr[t], acc);
            for (int t = kBndW<P>; t < L; ++t) acc = fmaT(a.W.lane(fam, i, t), Hr[t], acc);
        }
        sT[row * rT + i] = acc;
    }
}

}  // namespace stx
}  // namespace mfwq
