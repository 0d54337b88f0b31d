// Fused FP32 apply of Algorithm 2 (Section 3.2) for sm_103a.
//
// The staged FP32 apply writes the three trial partials Y = (B_3 (x) B_2) v
// and the nine test partials T^(ab) = W_1^(ab) (C_ab G_b) to HBM between its
// kernels (about 1.5 GB per apply at 196^3 DoFs, more than the coefficient
// itself).  Here one block owns a q3 plane (or a segment of its q2 lines) and
// sweeps it in batches of 8 q2 lines:
//   trial y : Y_b(q2, j1) = sum_j2 B2^(b)(q2, j2) Z(j2, j1) from a ring of Z rows
//             (Z0 = B0_3 v, Z1 = B1_3 v of this plane) in shared memory;
//   x stage : the stencil form of the staged kernel (stencil_x.cuh): G_b, the
//             products with the six coefficient fields, T^(ab) in shared memory;
//   test y  : U_g(i2, i1) += W2^(ab)(i2, q2) T^(ab)(q2, i1) into a ring of U rows,
//             g = 2 a3 + b3 the z family of (alpha, beta); a row leaves the
//             ring (to HBM) when its last weighted point has been swept.
// Only Z (in), the coefficient (in) and U (out) cross HBM; trial z and test z
// stay the slow-dimension kernels of the staged apply.
//
// A U row whose weight band crosses a segment boundary receives one partial
// sum from each of the two segments: both add it (red.global.add) onto a row
// zeroed just before the launch.  Two additions onto zero give the same value
// in either order, so the result does not depend on block scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "fused_apply.h"
#include "prof.h"
#include "stencil_x.cuh"

namespace mfwq {

namespace {

// q2b, nl, zlo, zhi, ulo, uhi, rlo, rhi, uniform, z0, u0, (pad): a uniform batch
// lies in direction 2's translation-invariant interior and runs the y
// contractions with the stencil taps of direction 2 on Z rows z0.. and U rows u0..
constexpr int kBatchInts = 12;

// Table widths the kernel is compiled for: a batch of 8 points of degree P
// reads at most P + 6 Z rows and touches at most P + 6 U rows (checked when
// the plan is built).
__host__ __device__ constexpr int fused_kmax(int P) { return P + 6; }

__host__ __device__ inline int odd_at_least(int n) { return n | 1; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// ------------------------------------------------------------------ host plan
namespace {

struct HostPlan {
    std::vector<int> batch, fp, lp, seg, straddle;
    std::vector<float> Bd, Wd;
};

// Direction-2 tables of the plan.  Returns false (with why) when a batch
// needs wider tables than the kernel holds or the row ranges are not
// contiguous (they are for every open knot vector: supports move monotonically).
bool build_batches(const Dir1D& d2, int P, HostPlan& hp, int& KZ, int& KU, int& maxsupp, std::string& why) {
    const Band1D& B = d2.B;   // rows q -> Z rows j2 (fams: values, derivatives)
    const Band1D& W = d2.W;   // rows i -> points q (4 fams)
    const int n2 = d2.n, nq2 = d2.nq, KM = fused_kmax(P);
    const int nbatch = (nq2 + kFusedLines - 1) / kFusedLines;
    hp.fp.assign(n2, 0);
    hp.lp.assign(n2, -1);
    maxsupp = 0;
    for (int i = 0; i < n2; ++i) {
        if (W.len[i] <= 0) {
            why = "a weight row without points";
            return false;
        }
        hp.fp[i] = W.start[i];
        hp.lp[i] = W.start[i] + W.len[i] - 1;
        maxsupp = std::max(maxsupp, W.len[i]);
        if (i > 0 && (hp.fp[i] < hp.fp[i - 1] || hp.lp[i] < hp.lp[i - 1])) {
            why = "weight bands not monotone";
            return false;
        }
    }
    hp.batch.assign((size_t)nbatch * kBatchInts, 0);
    hp.Bd.assign((size_t)nbatch * 2 * kFusedLines * KM, 0.f);
    hp.Wd.assign((size_t)nbatch * 4 * kFusedLines * KM, 0.f);
    KZ = KU = 0;
    for (int b = 0; b < nbatch; ++b) {
        const int q2b = b * kFusedLines, nl = std::min(kFusedLines, nq2 - q2b);
        int zlo = 1 << 30, zhi = -1;
        for (int l = 0; l < nl; ++l) {
            const int q = q2b + l;
            if (B.len[q] <= 0) continue;
            zlo = std::min(zlo, B.start[q]);
            zhi = std::max(zhi, B.start[q] + B.len[q]);
        }
        if (zhi < 0) zlo = zhi = 0;
        int ulo = -1, uhi = -1, rlo = -1, rhi = -1;
        for (int i = 0; i < n2; ++i) {
            const bool touch = hp.fp[i] <= q2b + nl - 1 && hp.lp[i] >= q2b;
            if (touch) {
                if (ulo < 0) ulo = i;
                if (uhi >= 0 && uhi != i) {
                    why = "U rows of a batch not contiguous";
                    return false;
                }
                uhi = i + 1;
            }
            const bool ret = hp.lp[i] >= q2b && hp.lp[i] < q2b + nl;
            if (ret) {
                if (rlo < 0) rlo = i;
                rhi = i + 1;
            }
        }
        if (ulo < 0) ulo = uhi = 0;
        if (rlo < 0) rlo = rhi = ulo;
        if (zhi - zlo > KM || uhi - ulo > KM) {
            why = "a batch needs more than P + 6 rows";
            return false;
        }
        KZ = std::max(KZ, zhi - zlo);
        KU = std::max(KU, uhi - ulo);
        int* bi = &hp.batch[(size_t)b * kBatchInts];
        bi[0] = q2b;
        bi[1] = nl;
        bi[2] = zlo;
        bi[3] = zhi;
        bi[4] = ulo;
        bi[5] = uhi;
        bi[6] = rlo;
        bi[7] = rhi;
        // dense B2 rows of the batch's points on Z rows zlo + k
        for (int f = 0; f < 2; ++f)
            for (int l = 0; l < nl; ++l) {
                const int q = q2b + l;
                for (int t = 0; t < B.len[q]; ++t) {
                    const int k = B.start[q] + t - zlo;
                    hp.Bd[(((size_t)b * 2 + f) * kFusedLines + l) * KM + k] = (float)B.at(f, q, t);
                }
            }
        // dense W2 of U rows ulo + k at the batch's points
        for (int f = 0; f < 4; ++f)
            for (int k = 0; k < uhi - ulo; ++k) {
                const int i = ulo + k;
                for (int t = 0; t < W.len[i]; ++t) {
                    const int q = W.start[i] + t;
                    if (q < q2b || q >= q2b + nl) continue;
                    hp.Wd[(((size_t)b * 4 + f) * kFusedLines + (q - q2b)) * KM + k] = (float)W.at(f, i, t);
                }
            }
    }
    // every row leaves the ring exactly once, right after it is last touched
    for (int b = 1; b < nbatch; ++b)
        if (hp.batch[(size_t)(b - 1) * kBatchInts + 7] != hp.batch[(size_t)b * kBatchInts + 4]) {
            why = "ring bookkeeping: retired rows do not meet the next batch's rows";
            return false;
        }
    return true;
}

// Flags the batches whose y contractions the stencil of direction 2 gives
// exactly: 8 points inside its invariant pair range, every U row the batch
// touches inside its invariant row range.  Their static windows: Z rows z0 +
// ((phi + l) >> 1) + t, t < P + 2, for point l; U rows u0 + k with tap
// t = psi + l + 2 (P - k) of the row filter.  Widens the U ring to hold them.
void flag_uniform(const Dir1D& d2, const StencilD<float>& S2, int P, HostPlan& hp, int& RU, int& phi, int& psi) {
    phi = psi = 0;
    if (!S2.ok || S2.P != P) return;
    phi = (S2.q_lo % 2 + 2) % 2;  // parity of (q2b - q_lo) for q2b a multiple of 8
    psi = (S2.qw % 2 + 2) % 2;
    const int nbatch = (int)(hp.batch.size() / kBatchInts);
    for (int b = 0; b < nbatch; ++b) {
        int* bi = &hp.batch[(size_t)b * kBatchInts];
        const int q2b = bi[0], nl = bi[1];
        if (nl != kFusedLines || q2b < S2.q_lo || q2b + kFusedLines > S2.q_hi) continue;
        const int K0 = (q2b - S2.q_lo - phi) / 2;
        const int z0 = S2.jb + K0;
        const int M = (q2b - S2.qw - psi) / 2;
        const int u0 = S2.i_lo + M - P;
        if (z0 < 0 || z0 > bi[2] || z0 + ((phi + 7) >> 1) + P + 2 < bi[3]) continue;
        if (u0 < S2.i_lo || u0 + P + 5 > S2.i_hi || bi[4] < u0 || bi[5] > u0 + P + 5) continue;
        bi[8] = 1;
        bi[9] = z0;
        bi[10] = u0;
        RU = std::max(RU, std::max(bi[5], u0 + P + 5) - std::min(bi[4], u0));
    }
    (void)d2;
}

}  // namespace

// ------------------------------------------------------------------ device
namespace {

using stx::kStLines;
static_assert(kStLines == kFusedLines, "the fused batch is the stencil x stage's block of lines");
static_assert(kFusedThreads == kThreads, "the stencil x stage runs on 256 threads");

struct FusedArgs {
    XArgs<float> x;          // direction 1: tables, coefficient, n1, nq1
    StencilD<float> st;      // direction 1: translation-invariant interior
    const int* batch;        // plan tables (FusedPlan)
    const float* Bd;
    const float* Wd;
    const int* fp;
    const int* lp;
    const int* seg;
    const float* z0;         // Z0, Z1 [nq3][n2][n1]
    const float* z1;
    float* u;                // U_g at u + g * us, [nq3][n2][n1]
    size_t us;
    int n2, nq2, S, items, RZ, RU, rY, rG, rT;
    int phi, psi;            // phases of the uniform batches (see flag_uniform)
    const int* skip;
    StencilD<float> st2;     // direction 2: taps of the uniform batches
    CoeffField cf;           // the coefficient evaluated in the block (ONF kernels)
};

// U rows that two segments share start at zero (both segments add into them).
__global__ void k_fused_zero(float* __restrict__ u, size_t us, const int* __restrict__ rows, int nrows, int n1, int n2,
                             int nq3, const int* skip) {
    if (skip && *skip) return;
    const size_t per_g = (size_t)nq3 * nrows * n1;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < 4 * per_g; e += (size_t)gridDim.x * blockDim.x) {
        const size_t g = e / per_g, r = e - g * per_g;
        const size_t q3 = r / ((size_t)nrows * n1), rr = r - q3 * nrows * n1;
        const int k = (int)(rr / n1), i = (int)(rr - (size_t)k * n1);
        u[g * us + ((size_t)q3 * n2 + rows[k]) * n1 + i] = 0.f;
    }
}

// Every access to the Z and U rings is owned by one thread (column j or i is
// thread j mod 256 in every phase), so the rings need no barriers.

// Trial y of one beta: Y_b(l, j1) = sum_k B2^(fam)(q2b + l, zlo + k) Z(zlo + k, j1)
// for the batch's 8 lines, into sY.  Z family: Z1 = B1_3 v for beta = 3, else Z0;
// B2 family: derivative for beta = 2.
template <int P, int BETA>
__device__ __forceinline__ void fa_trial_y(const FusedArgs& a, const float* __restrict__ Bd, int zlo, int nkz,
                                           const float* sZ, float* sY) {
    constexpr int KM = fused_kmax(P);
    constexpr int FB = BETA == 1 ? 1 : 0;
    constexpr int ZB = BETA == 2 ? 1 : 0;
    const int n1 = a.x.n1, RZ = a.RZ;
    const float* zr = sZ + (size_t)ZB * RZ * n1;
    const float* w = Bd + FB * kFusedLines * KM;
    const int s0 = zlo % RZ;
    for (int j = threadIdx.x; j < n1; j += kFusedThreads) {
        float z[KM];
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            z[k] = 0.f;
            if (k < nkz) {
                int slot = s0 + k;
                if (slot >= RZ) slot -= RZ;
                z[k] = zr[slot * n1 + j];
            }
        }
#pragma unroll
        for (int l = 0; l < kFusedLines; ++l) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < KM; ++k) acc = fmaf(__ldg(w + l * KM + k), z[k], acc);
            sY[l * a.rY + j] = acc;
        }
    }
}

// Test y of one beta: for the three T^(alpha beta) rows of every line,
// U_g(ulo + k, i1) += sum_l W2^(a2 b2)(ulo + k, q2b + l) T^(alpha beta)(l, i1),
// g = 2 [alpha = 3] + [beta = 3], (a2, b2) = ([alpha = 2], [beta = 2]).  The
// two z groups of a beta (alpha = 1, 2 and alpha = 3) are summed one after the
// other, so only one group's accumulators are live.
template <int P, int BETA, int AL0, int AL1>
__device__ __forceinline__ void fa_test_y_group(const FusedArgs& a, const float* __restrict__ Wd, int ulo, int nku,
                                                int nl, int i, const float* sT, float* sU) {
    constexpr int KM = fused_kmax(P);
    constexpr int G = 2 * (AL0 == 2 ? 1 : 0) + (BETA == 2 ? 1 : 0);
    const int n1 = a.x.n1, RU = a.RU;
    float acc[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) acc[k] = 0.f;
#pragma unroll
    for (int al = AL0; al <= AL1; ++al) {
        const int fam = 2 * (al == 1 ? 1 : 0) + (BETA == 1 ? 1 : 0);
        const float* w = Wd + fam * kFusedLines * KM;
#pragma unroll
        for (int l = 0; l < kFusedLines; ++l) {
            const float t = l < nl ? sT[(al * kFusedLines + l) * a.rT + i] : 0.f;
#pragma unroll
            for (int k = 0; k < KM; ++k) acc[k] = fmaf(__ldg(w + l * KM + k), t, acc[k]);
        }
    }
    int slot = ulo % RU;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (k < nku) sU[(G * RU + slot) * n1 + i] += acc[k];
        if (++slot == RU) slot = 0;
    }
}

template <int P, int BETA>
__device__ __forceinline__ void fa_test_y(const FusedArgs& a, const float* __restrict__ Wd, int ulo, int nku, int nl,
                                          const float* sT, float* sU) {
    for (int i = threadIdx.x; i < a.x.n1; i += kFusedThreads) {
        fa_test_y_group<P, BETA, 0, 1>(a, Wd, ulo, nku, nl, i, sT, sU);
        fa_test_y_group<P, BETA, 2, 2>(a, Wd, ulo, nku, nl, i, sT, sU);
    }
}

// The same two phases for a uniform batch: the taps are direction 2's stencil
// filters (kernel parameters, compile-time indices, no zero taps).
// Trial: point l (phase (PHI + l) & 1 of its pair) reads Z rows
// z0 + ((PHI + l) >> 1) + t, t < P + 2.
template <int P, int BETA, int PHI>
__device__ __forceinline__ void fa_trial_y_st(const FusedArgs& a, int z0, const float* sZ, float* sY) {
    constexpr int FB = BETA == 1 ? 1 : 0;
    constexpr int ZB = BETA == 2 ? 1 : 0;
    constexpr int NZ = ((PHI + kFusedLines - 1) >> 1) + P + 2;
    const int n1 = a.x.n1, RZ = a.RZ;
    const float* zr = sZ + (size_t)ZB * RZ * n1;
    const int s0 = z0 % RZ;
    for (int j = threadIdx.x; j < n1; j += kFusedThreads) {
        float z[NZ];
        int slot = s0;
#pragma unroll
        for (int k = 0; k < NZ; ++k) {
            z[k] = zr[slot * n1 + j];
            if (++slot == RZ) slot = 0;
        }
#pragma unroll
        for (int l = 0; l < kFusedLines; ++l) {
            const int ph = (PHI + l) & 1, o = (PHI + l) >> 1;
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t < P + 2; ++t) acc = fmaf(a.st2.bf[FB][ph][t], z[o + t], acc);
            sY[l * a.rY + j] = acc;
        }
    }
}

// Test: point l reaches U row u0 + k through tap t = PSI + l + 2 (P - k) of the
// row filter (0 <= t <= 2P).
template <int P, int BETA, int PSI, int AL0, int AL1>
__device__ __forceinline__ void fa_test_y_st_group(const FusedArgs& a, int u0, int i, const float* sT, float* sU) {
    constexpr int NU = P + 5;
    constexpr int G = 2 * (AL0 == 2 ? 1 : 0) + (BETA == 2 ? 1 : 0);
    const int n1 = a.x.n1, RU = a.RU;
    float acc[NU];
#pragma unroll
    for (int k = 0; k < NU; ++k) acc[k] = 0.f;
#pragma unroll
    for (int al = AL0; al <= AL1; ++al) {
        const int fam = 2 * (al == 1 ? 1 : 0) + (BETA == 1 ? 1 : 0);
#pragma unroll
        for (int l = 0; l < kFusedLines; ++l) {
            const float t = sT[(al * kFusedLines + l) * a.rT + i];
#pragma unroll
            for (int k = 0; k < NU; ++k) {
                const int tap = PSI + l + 2 * (P - k);
                if (tap >= 0 && tap <= 2 * P) acc[k] = fmaf(a.st2.wf[fam][tap], t, acc[k]);
            }
        }
    }
    int slot = u0 % RU;
#pragma unroll
    for (int k = 0; k < NU; ++k) {
        sU[(G * RU + slot) * n1 + i] += acc[k];
        if (++slot == RU) slot = 0;
    }
}

template <int P, int BETA, int PSI>
__device__ __forceinline__ void fa_test_y_st(const FusedArgs& a, int u0, const float* sT, float* sU) {
    for (int i = threadIdx.x; i < a.x.n1; i += kFusedThreads) {
        fa_test_y_st_group<P, BETA, PSI, 0, 1>(a, u0, i, sT, sU);
        fa_test_y_st_group<P, BETA, PSI, 2, 2>(a, u0, i, sT, sU);
    }
}

// Rows r0 .. r1-1 leave the ring: to U by a plain store when the row's whole
// weight band lies in this segment's points [qa, qb), else by an atomic add
// (the row is shared with a neighbouring segment); their slots are cleared.
__device__ __forceinline__ void fa_retire(const FusedArgs& a, int q3, int r0, int r1, int qa, int qb, bool force_add,
                                          float* sU) {
    const int n1 = a.x.n1, RU = a.RU;
    for (int r = r0; r < r1; ++r) {
        const int slot = r % RU;
        const bool owned = !force_add && a.fp[r] >= qa && a.lp[r] < qb;
        float* dst0 = a.u + ((size_t)q3 * a.n2 + r) * n1;
        for (int i = threadIdx.x; i < n1; i += kFusedThreads) {
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float* src = sU + (g * RU + slot) * n1 + i;
                const float v = *src;
                *src = 0.f;
                float* dst = dst0 + g * a.us + i;
                if (owned) *dst = v;
                else atomicAdd(dst, v);
            }
        }
    }
}

// One beta of a batch: trial y -> x-stage trial -> x-stage test -> test y.
template <int P, int BETA, bool ONF>
__device__ __forceinline__ void fa_beta(const FusedArgs& a, const int* bi, int line0, const float* Bd, const float* Wd,
                                        float* sY, float* sH, float* sT, const float* sZ, float* sU, const float* sK) {
    const int nl = bi[1];
    const bool uni = bi[8] != 0;
    if (!uni) fa_trial_y<P, BETA>(a, Bd, bi[2], bi[3] - bi[2], sZ, sY);
    else if (a.phi) fa_trial_y_st<P, BETA, 1>(a, bi[9], sZ, sY);
    else fa_trial_y_st<P, BETA, 0>(a, bi[9], sZ, sY);
    __syncthreads();
    if (ONF) stx::st_trial_otf<P, BETA>(a.x, a.st, nl, sY, sH, a.rY, a.rG, sK, a.rG, a.cf.g6);
    else stx::st_trial<float, P, BETA>(a.x, a.st, line0, nl, sY, sH, a.rY, a.rG);
    __syncthreads();
    stx::st_test<float, P, BETA>(a.x, a.st, sH, sT, a.rG, a.rT);
    __syncthreads();
    if (!uni) fa_test_y<P, BETA>(a, Wd, bi[4], bi[5] - bi[4], nl, sT, sU);
    else if (a.psi) fa_test_y_st<P, BETA, 1>(a, bi[10], sT, sU);
    else fa_test_y_st<P, BETA, 0>(a, bi[10], sT, sU);
}

template <int P, bool ONF>
__global__ void __launch_bounds__(kFusedThreads, 2) k_apply_fused(FusedArgs a) {
    if (a.skip && *a.skip) return;
    constexpr int KM = fused_kmax(P);
    extern __shared__ __align__(16) unsigned char fsm[];
    const int n1 = a.x.n1, nq1 = a.x.nq1;
    float* sH = reinterpret_cast<float*>(fsm);                  // [3 alpha][8][rG]
    float* sT = sH + 3 * kFusedLines * a.rG;                     // [3 alpha][8][rT]
    float* sY = sT;                                              // [8][rY]: the alpha = 1 slab of sT (rY = rT)
    float* sZ = sT + 3 * kFusedLines * a.rT;                     // [2][RZ][n1]
    float* sU = sZ + 2 * a.RZ * n1;                              // [4][RU][n1]
    float* sK = sU + 4 * a.RU * n1;                              // ONF: [8][rG] kappa of the batch's lines
    float* sAB = sK + kFusedLines * a.rG;                        // ONF: [8][kMaxModes][4]
    // both rings start at zero: zero taps of a uniform batch may read Z slots
    // no row was loaded into, and must not meet a NaN pattern there
    for (int i = threadIdx.x; i < n1; i += kFusedThreads) {
        for (int r = 0; r < 4 * a.RU; ++r) sU[r * n1 + i] = 0.f;
        for (int r = 0; r < 2 * a.RZ; ++r) sZ[r * n1 + i] = 0.f;
    }
    for (int item = blockIdx.x; item < a.items; item += gridDim.x) {
        const int q3 = item / a.S, s = item - q3 * a.S;
        const int b0 = a.seg[2 * s], b1 = a.seg[2 * s + 1];
        const int qa = b0 * kFusedLines, qb = min(b1 * kFusedLines, a.nq2);
        int zloaded = -1;  // Z rows below zloaded are in the ring
        for (int b = b0; b < b1; ++b) {
            const int* bi = a.batch + (size_t)b * kBatchInts;
            const int q2b = bi[0], nl = bi[1], zlo = bi[2], zhi = bi[3];
            const int line0 = q3 * a.nq2 + q2b;
            // coefficient rows into L2 ahead of use: at a segment's start its
            // first two batches, then always the batch after next
            if (!ONF && threadIdx.x < 12) {
                const int f = threadIdx.x % 6, ahead = threadIdx.x / 6;  // 0: batch b + 2, 1: batch b (segment start)
                const int bp = ahead ? b : b + 2;
                if ((ahead == 0 || b == b0) && bp < b1) {
                    const int q = bp * kFusedLines, n = min(kFusedLines, a.nq2 - q);
                    ptx::prefetch_l2_range(a.x.C + (size_t)f * a.x.cs + ((size_t)q3 * a.nq2 + q) * nq1,
                                           sizeof(float) * (size_t)n * nq1);
                }
                if (ahead == 0 && b == b0 && b + 1 < b1) {
                    const int q = (b + 1) * kFusedLines, n = min(kFusedLines, a.nq2 - q);
                    ptx::prefetch_l2_range(a.x.C + (size_t)f * a.x.cs + ((size_t)q3 * a.nq2 + q) * nq1,
                                           sizeof(float) * (size_t)n * nq1);
                }
            }
            // new Z rows of this batch (column-owned)
            const float* z0p = a.z0 + (size_t)q3 * a.n2 * n1;
            const float* z1p = a.z1 + (size_t)q3 * a.n2 * n1;
            for (int r = max(zlo, zloaded); r < zhi; ++r) {
                const int slot = r % a.RZ;
                for (int j = threadIdx.x; j < n1; j += kFusedThreads) {
                    sZ[slot * n1 + j] = z0p[(size_t)r * n1 + j];
                    sZ[(a.RZ + slot) * n1 + j] = z1p[(size_t)r * n1 + j];
                }
            }
            zloaded = zhi;
            const float* Bd = a.Bd + (size_t)b * 2 * kFusedLines * KM;
            const float* Wd = a.Wd + (size_t)b * 4 * kFusedLines * KM;
            if (ONF) stx::st_kappa(a.cf, line0, nl, nq1, a.nq2, sK, a.rG, sAB);
            fa_beta<P, 0, ONF>(a, bi, line0, Bd, Wd, sY, sH, sT, sZ, sU, sK);
            fa_beta<P, 1, ONF>(a, bi, line0, Bd, Wd, sY, sH, sT, sZ, sU, sK);
            fa_beta<P, 2, ONF>(a, bi, line0, Bd, Wd, sY, sH, sT, sZ, sU, sK);
            fa_retire(a, q3, bi[6], bi[7], qa, qb, false, sU);
            if (b + 1 == b1) fa_retire(a, q3, bi[7], bi[5], qa, qb, true, sU);  // rows that continue in the next segment
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ host launch
namespace {

template <int P>
void launch_p(const FusedPlan& pl, const FusedArgs& a, bool onf, cudaStream_t s) {
    if (onf) k_apply_fused<P, true><<<pl.grid, kFusedThreads, pl.smem_onf, s>>>(a);
    else k_apply_fused<P, false><<<pl.grid, kFusedThreads, pl.smem, s>>>(a);
}

template <int P>
cudaError_t occupancy_p(int smem, int* blocks) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_apply_fused<P, false>, kFusedThreads, smem);
}

cudaError_t occupancy(int P, int smem, int* blocks) {
    switch (P) {
        case 2: return occupancy_p<2>(smem, blocks);
        case 3: return occupancy_p<3>(smem, blocks);
        case 4: return occupancy_p<4>(smem, blocks);
        case 5: return occupancy_p<5>(smem, blocks);
        case 6: return occupancy_p<6>(smem, blocks);
        case 7: return occupancy_p<7>(smem, blocks);
        case 8: return occupancy_p<8>(smem, blocks);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// The dynamic shared-memory limit is a per-kernel attribute shared by all
// handles on a device, so it only ever grows (one record per device).
int configure_fused_smem(int bytes) {
    static std::mutex mu;
    static int configured[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MFWQ_ECUDA;
    std::lock_guard<std::mutex> lk(mu);
    if (bytes <= configured[dev]) return MFWQ_OK;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, A, bytes);
    };
    set(k_apply_fused<2, false>);
    set(k_apply_fused<3, false>);
    set(k_apply_fused<4, false>);
    set(k_apply_fused<5, false>);
    set(k_apply_fused<6, false>);
    set(k_apply_fused<7, false>);
    set(k_apply_fused<8, false>);
    set(k_apply_fused<2, true>);
    set(k_apply_fused<3, true>);
    set(k_apply_fused<4, true>);
    set(k_apply_fused<5, true>);
    set(k_apply_fused<6, true>);
    set(k_apply_fused<7, true>);
    set(k_apply_fused<8, true>);
    if (e != cudaSuccess) return MFWQ_ECUDA;
    configured[dev] = bytes;
    return MFWQ_OK;
}

int fused_plan_build(const Dir1D& d1, const Dir1D& d2, const StencilD<float>& S1, const StencilD<float>& S2, int nq3,
                     FusedPlan& pl) {
    fused_plan_free(pl);
    pl.ok = 0;
    if (!S1.ok || S1.P < 2 || S1.P > kStencilMaxP) {
        pl.why = "direction 1 has no translation-invariant interior (non-uniform knots or degree above 8)";
        return MFWQ_OK;
    }
    const int P = S1.P, KM = fused_kmax(P);
    HostPlan hp;
    int KZ = 0, KU = 0, maxsupp = 0;
    if (!build_batches(d2, P, hp, KZ, KU, maxsupp, pl.why)) return MFWQ_OK;
    const int n1 = d1.n, nq1 = d1.nq, nbatch = (d2.nq + kFusedLines - 1) / kFusedLines;
    pl.P = P;
    pl.nbatch = nbatch;
    pl.KZ = KZ;
    pl.KU = KU;
    int RU = KU;
    flag_uniform(d2, S2, P, hp, RU, pl.phi, pl.psi);
    pl.nuniform = 0;
    for (size_t b = 0; b < hp.batch.size() / kBatchInts; ++b) pl.nuniform += hp.batch[b * kBatchInts + 8];
    pl.RZ = std::max(1, KZ);
    pl.RU = std::max(1, RU);
    pl.rY = pl.rT = odd_at_least(n1);
    pl.rG = odd_at_least(nq1);
    const size_t floats = (size_t)3 * kFusedLines * pl.rG + (size_t)3 * kFusedLines * pl.rT + (size_t)2 * pl.RZ * n1 +
                          (size_t)4 * pl.RU * n1;
    if (floats * sizeof(float) > (size_t)kXstageSmemMax) {
        pl.why = "shared memory of a block would exceed 227 KB";
        return MFWQ_OK;
    }
    pl.smem = (int)(floats * sizeof(float));
    pl.smem_onf = (int)((floats + (size_t)kFusedLines * pl.rG + (size_t)kFusedLines * kMaxModes * 4) * sizeof(float));
    int st = configure_fused_smem(std::min(pl.smem_onf, kXstageSmemMax));
    if (st != MFWQ_OK) return st;
    int dev = 0, sms = 0, bps = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        occupancy(P, pl.smem, &bps) != cudaSuccess || bps < 1) {
        cudaGetLastError();
        pl.why = "occupancy query failed";
        return MFWQ_OK;
    }
    const int resident = sms * bps;
    // segments: enough work items for about four per resident block, each
    // segment at least one weight band long (a row spans at most two segments)
    const int min_batches = std::max(1, (maxsupp + kFusedLines - 1) / kFusedLines);
    const int smax = std::max(1, nbatch / min_batches);
    int S = (4 * resident + nq3 - 1) / std::max(1, nq3);
    S = std::max(1, std::min(S, smax));
    pl.S = S;
    hp.seg.resize(2 * S);
    for (int s = 0; s < S; ++s) {
        hp.seg[2 * s] = (int)((long long)s * nbatch / S);
        hp.seg[2 * s + 1] = (int)((long long)(s + 1) * nbatch / S);
    }
    for (int s = 0; s < S; ++s)
        if ((hp.seg[2 * s + 1] - hp.seg[2 * s]) * kFusedLines < maxsupp && S > 1) {
            pl.why = "segment shorter than a weight band";
            return MFWQ_OK;
        }
    for (int i = 0; i < d2.n; ++i)
        for (int s = 1; s < S; ++s) {
            const int qa = hp.seg[2 * s] * kFusedLines;
            if (hp.fp[i] < qa && hp.lp[i] >= qa) {
                hp.straddle.push_back(i);
                break;
            }
        }
    pl.nstraddle = (int)hp.straddle.size();
    const long long items = (long long)nq3 * S;
    pl.grid = (int)std::min<long long>(items, resident);
    // device tables
    size_t off = 0;
    const size_t o_batch = off;
    off = align256(off + hp.batch.size() * sizeof(int));
    const size_t o_fp = off;
    off = align256(off + hp.fp.size() * sizeof(int));
    const size_t o_lp = off;
    off = align256(off + hp.lp.size() * sizeof(int));
    const size_t o_seg = off;
    off = align256(off + hp.seg.size() * sizeof(int));
    const size_t o_str = off;
    off = align256(off + std::max<size_t>(1, hp.straddle.size()) * sizeof(int));
    const size_t o_bd = off;
    off = align256(off + hp.Bd.size() * sizeof(float));
    const size_t o_wd = off;
    off = align256(off + hp.Wd.size() * sizeof(float));
    std::vector<unsigned char> host(off, 0);
    std::memcpy(host.data() + o_batch, hp.batch.data(), hp.batch.size() * sizeof(int));
    std::memcpy(host.data() + o_fp, hp.fp.data(), hp.fp.size() * sizeof(int));
    std::memcpy(host.data() + o_lp, hp.lp.data(), hp.lp.size() * sizeof(int));
    std::memcpy(host.data() + o_seg, hp.seg.data(), hp.seg.size() * sizeof(int));
    if (!hp.straddle.empty()) std::memcpy(host.data() + o_str, hp.straddle.data(), hp.straddle.size() * sizeof(int));
    std::memcpy(host.data() + o_bd, hp.Bd.data(), hp.Bd.size() * sizeof(float));
    std::memcpy(host.data() + o_wd, hp.Wd.data(), hp.Wd.size() * sizeof(float));
    if (cudaMalloc(&pl.dmem, off) != cudaSuccess) {
        cudaGetLastError();
        pl.dmem = nullptr;
        return MFWQ_ENOMEM;
    }
    if (cudaMemcpy(pl.dmem, host.data(), off, cudaMemcpyHostToDevice) != cudaSuccess) return MFWQ_ECUDA;
    unsigned char* base = static_cast<unsigned char*>(pl.dmem);
    pl.batch = reinterpret_cast<const int*>(base + o_batch);
    pl.fp = reinterpret_cast<const int*>(base + o_fp);
    pl.lp = reinterpret_cast<const int*>(base + o_lp);
    pl.seg = reinterpret_cast<const int*>(base + o_seg);
    pl.straddle = reinterpret_cast<const int*>(base + o_str);
    pl.Bd = reinterpret_cast<const float*>(base + o_bd);
    pl.Wd = reinterpret_cast<const float*>(base + o_wd);
    (void)KM;
    pl.ok = 1;
    pl.why.clear();
    return MFWQ_OK;
}

void fused_plan_free(FusedPlan& pl) {
    if (pl.dmem) cudaFree(pl.dmem);
    pl.dmem = nullptr;
    pl.ok = 0;
}

cudaError_t launch_fused(const OpCtx<float>& c, const FusedPlan& pl, const float* z0, const float* z1, float* u,
                         size_t us, const int* skip) {
    const DirD<float>& d1 = c.d[0];
    const DirD<float>& d2 = c.d[1];
    const DirD<float>& d3 = c.d[2];
    FusedArgs a;
    a.x = xargs(d1, d3.nq * d2.nq, c.cs, c.C);
    a.st = d1.SX;
    a.batch = pl.batch;
    a.Bd = pl.Bd;
    a.Wd = pl.Wd;
    a.fp = pl.fp;
    a.lp = pl.lp;
    a.seg = pl.seg;
    a.z0 = z0;
    a.z1 = z1;
    a.u = u;
    a.us = us;
    a.n2 = d2.n;
    a.nq2 = d2.nq;
    a.S = pl.S;
    a.items = d3.nq * pl.S;
    a.RZ = pl.RZ;
    a.RU = pl.RU;
    a.rY = pl.rY;
    a.rG = pl.rG;
    a.rT = pl.rT;
    a.phi = pl.phi;
    a.psi = pl.psi;
    a.skip = skip;
    a.st2 = d2.SX;
    if (pl.nstraddle > 0) {
        const size_t n = (size_t)4 * d3.nq * pl.nstraddle * d1.n;
        const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 4096);
        launch_begin(S_FUSED, c.stream);
        k_fused_zero<<<blocks, 256, 0, c.stream>>>(u, us, pl.straddle, pl.nstraddle, d1.n, d2.n, d3.nq, skip);
        launch_end(S_FUSED, c.stream);
    }
    launch_begin(S_FUSED, c.stream);
    const bool onf = c.cf != nullptr;
    if (onf) {
        if (pl.smem_onf > kXstageSmemMax) return cudaErrorInvalidValue;
        a.cf = *c.cf;
    }
    switch (pl.P) {
        case 2: launch_p<2>(pl, a, onf, c.stream); break;
        case 3: launch_p<3>(pl, a, onf, c.stream); break;
        case 4: launch_p<4>(pl, a, onf, c.stream); break;
        case 5: launch_p<5>(pl, a, onf, c.stream); break;
        case 6: launch_p<6>(pl, a, onf, c.stream); break;
        case 7: launch_p<7>(pl, a, onf, c.stream); break;
        case 8: launch_p<8>(pl, a, onf, c.stream); break;
        default: break;  // unreachable: plans exist only for P in 2..8
    }
    launch_end(S_FUSED, c.stream);
    return cudaGetLastError();
}

}  // namespace mfwq
