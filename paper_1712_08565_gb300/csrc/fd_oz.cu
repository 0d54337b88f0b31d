// FP64-accurate FD mode products on the BF16 tensor cores by operand
// splitting (see fd_oz.h for the scheme and its error bound).
//
// One pass contracts the fastest dimension of its input and writes the new
// index as the slowest dimension of its output, as the TF32/BF16 passes of
// fd_tc.cu do:  D[r][o] = sum_t A[r][t] Bm[o][t],  Out[o][r] = D[r][o].
//
// A CTA (256 threads, one per SM: its TMEM blocks take the 512 columns) computes 128 rows x kOzNT outputs of one pass per work item.
//  * Row exponents: the largest biased exponent of each of its 128 rows of A.
//  * Per K chunk of 32 elements (two pipeline stages): thread 0 starts the
//    bulk copy of the precomputed Bm slices of the chunk; all threads read A
//    (two threads per row, 16 elements each), split each element into its 7
//    slices with integer operations and store them as BF16 in the MMA layout;
//    then thread 0 issues the 36 slice-pair products (two K steps each) into
//    the TMEM block of their level and commits to the stage's mbarrier.
//  * Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and half the
//    columns; per output the 8 level sums (integers in FP32) are converted to
//    integers, added with their weights 2^(7 (9 - L)) in 128 bits and rounded
//    to FP64 by constructing the bit pattern with the row and column scales;
//    the scaling pass multiplies by 1 / (lam1 + lam2 + lam3) from a table.
// Every mbarrier wait is bounded; on timeout the kernel records an error,
// waits (bounded) for its copies and products in flight, frees TMEM and
// returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "fd_oz.h"
#include "grouped.h"
#include "kernels.h"
#include "prof.h"
#include "ptx_async.cuh"

namespace mfwq {
namespace {

using ptx::mbar_expect_tx;
using ptx::mbar_init;
using ptx::mbar_wait;
using ptx::smem_u32;

constexpr int kOzThreads = 256;
constexpr int kOzTileM = 128;
constexpr int kOzSliceA = kOzTileM * kOzKC * 2;    // bytes of one A slice tile (8 KB)
constexpr int kOzSliceB = kOzNT * kOzKC * 2;       // bytes of one Bm slice tile (4 KB)
constexpr int kOzStageA = kOzSlices * kOzSliceA;   // 56 KB
constexpr int kOzStageB = kOzSlices * kOzSliceB;   // 28 KB
constexpr int kOzStage = kOzStageA + kOzStageB;
constexpr int kOzStages = 2;
constexpr int kOzTmemCols = 512;                   // kOzLevels * kOzNT
constexpr int kOzSmem = kOzStages * kOzStage + 1024 /* alignment */ + 64 /* barriers */ + 2 * kOzTileM * 4;

static_assert(kOzLevels * kOzNT <= kOzTmemCols, "level accumulators exceed TMEM");
static_assert(kOzSlices == 8 && kOzBits == 7, "the slice extraction below is written for 8 x 7 bits");

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; base offset 0, no swizzle
    return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128.
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kOzTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive TMEM columns of this warp's 32 lanes (no wait).
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// BF16 bit patterns of +-a (0 <= a < 2^7) for two elements, packed (element
// k in the low half): a + 2^23 is formed exactly from the bits, the FMA with
// the sign removes 2^23 exactly, and a value of at most 8 significant bits
// has a zero low half in FP32.
__device__ __forceinline__ uint32_t oz_pack2(uint32_t a0, float sg0, float c0, uint32_t a1, float sg1, float c1) {
    const float f0 = fmaf(sg0, __uint_as_float(0x4B000000u | a0), c0);
    const float f1 = fmaf(sg1, __uint_as_float(0x4B000000u | a1), c1);
    return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// Slice s (0 .. 7) of a 56-bit fixed-point magnitude held as (xh, xl) =
// (bits 32..55, bits 0..31): bits [49 - 7 s, 56 - 7 s).
template <int S>
__device__ __forceinline__ uint32_t oz_slice(uint32_t xh, uint32_t xl) {
    constexpr int lo = kOzFix - kOzBits * (S + 1);
    if constexpr (lo >= 32) return (xh >> (lo - 32)) & 127u;
    else if constexpr (lo + 7 <= 32) return (xl >> lo) & 127u;
    else return __funnelshift_r(xl, xh, lo) & 127u;
}

// The FP64 value of sum_L v[L - 2] 2^(7 (9 - L)) 2^(scale - 2107), L = 2 .. 9,
// v the level sums (integers held in FP32): 128-bit integer sum, rounded to
// 53 bits (half up on the magnitude), bit pattern built directly.
__device__ __forceinline__ double oz_combine(const float* v, int scale) {
    long long iv[kOzLevels];
#pragma unroll
    for (int l = 0; l < kOzLevels; ++l) iv[l] = __float2int_rn(v[l]);
    const long long hi = (iv[0] << 21) + (iv[1] << 14) + (iv[2] << 7) + iv[3];  // |hi| < 2^44
    const long long lo = (iv[4] << 21) + (iv[5] << 14) + (iv[6] << 7) + iv[7];  // |lo| < 2^47
    // T = hi 2^28 + lo as (th, tl), two's complement
    unsigned long long tl = (unsigned long long)hi << 28;
    long long th = hi >> 36;
    const unsigned long long t2 = tl + (unsigned long long)lo;
    th += (lo >> 63) + (t2 < tl ? 1 : 0);
    tl = t2;
    const bool neg = th < 0;
    if (neg) {
        tl = ~tl + 1ull;
        th = ~th + (tl == 0ull ? 1 : 0);
    }
    int adj = 0;
    unsigned long long M = tl;
    if (th != 0) {  // |T| < 2^73: keep the top 64 bits
        adj = 64 - __clzll(th);
        M = ((unsigned long long)th << (64 - adj)) | (tl >> adj);
    }
    if (M == 0ull) return 0.0;
    int msb = 63 - __clzll((long long)M);
    unsigned long long mant;
    if (msb > 52) {
        const int sh = msb - 52;
        mant = (M >> sh) + ((M >> (sh - 1)) & 1ull);
        if (mant >> 53) {
            mant >>= 1;
            ++msb;
        }
    } else {
        mant = M << (52 - msb);
    }
    const int E = msb + adj + scale - 2107 + 1023;
    if (E <= 0) return 0.0;
    const unsigned long long bits = ((unsigned long long)(neg ? 1 : 0) << 63) |
                                    ((unsigned long long)(E < 2047 ? E : 2047) << 52) |
                                    (E < 2047 ? (mant & 0xFFFFFFFFFFFFFull) : 0ull);
    return __longlong_as_double((long long)bits);
}

struct OzArgs {
    const double* A;     // [R][n_in]
    double* Out;         // [n_out][R]
    OzMat B;
    const double* dinv;  // null, or the [n_out][R] scaling table
    int R;
    int* err;
    const int* skip;
};

__global__ void __launch_bounds__(kOzThreads, 1) k_fd_oz(OzArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOzStages * kOzStage);  // Bm slices arrived
    uint64_t* done = full + kOzStages;                                          // the stage's products finished
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + kOzStages);
    int* s_e = reinterpret_cast<int*>(smem + kOzStages * kOzStage + 64);        // [2][128] row exponents
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kOzTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kOzStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&done[s]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int n_in = a.B.n_in, n_out = a.B.n_out, kch = a.B.k_chunks, ntl = a.B.n_tiles;
    const int mtiles = (a.R + kOzTileM - 1) / kOzTileM;
    const int items = mtiles * ntl;
    const int r = tid & (kOzTileM - 1), half = tid >> 7;  // slicing: row r, elements 16 half .. 16 half + 15
    bool ok = true;
    int g = 0;       // chunks consumed by this CTA (stage g & 1, use g >> 1)
    int issued = 0;     // Bm copies started (thread 0)
    int committed = 0;  // chunks whose products were committed (thread 0)
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const int mt = item / ntl, nt = item - mt * ntl;
        const int row0 = mt * kOzTileM;
        const int row = row0 + r;
        const double* Arow = a.A + (size_t)(row < a.R ? row : 0) * n_in;
        // largest biased exponent of each row (two threads per row)
        {
            int e = 0;
            if (row < a.R)
                for (int t = half; t < n_in; t += 2)
                    e = max(e, (int)((__double_as_longlong(__ldg(Arow + t)) >> 52) & 0x7FF));
            s_e[half * kOzTileM + r] = e;
        }
        __syncthreads();
        const int emax = max(s_e[r], s_e[kOzTileM + r]);
        const int nvalid = min(kOzNT, n_out - nt * kOzNT);
        const int nmma = (nvalid + 15) & ~15;
        const uint32_t idesc = idesc_bf16(nmma);
        for (int c = 0; c < kch; ++c, ++g) {
            const int s = g & 1, use = g >> 1;
            unsigned char* sa = smem + s * kOzStage;
            unsigned char* sb = sa + kOzStageA;
            {  // the stage's previous products must have finished (every thread leaves together on a timeout)
                const bool w = use < 1 || mbar_wait(smem_u32(&done[s]), (uint32_t)((use - 1) & 1));
                if (!__syncthreads_and(w ? 1 : 0)) {
                    ok = false;
                    break;
                }
            }
            if (tid == 0) {
                mbar_expect_tx(smem_u32(&full[s]), (uint32_t)kOzStageB);
                ptx::bulk_g2s(smem_u32(sb), a.B.sl + ((size_t)nt * kch + c) * (kOzStageB / 2), (uint32_t)kOzStageB,
                              smem_u32(&full[s]));
                ++issued;
            }
            // A: 16 elements of row r, split into 7 BF16 slices each
            uint32_t xh[16], xl[16];
            float sg[16], sc[16];
            const int k0 = c * kOzKC + 16 * half;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int k = k0 + i;
                const unsigned long long b =
                    (row < a.R && k < n_in) ? (unsigned long long)__double_as_longlong(__ldg(Arow + k)) : 0ull;
                const uint64_t X = oz_fixed(b, emax);
                xh[i] = (uint32_t)(X >> 32);
                xl[i] = (uint32_t)X;
                const bool ng = (b >> 63) != 0ull;
                sg[i] = ng ? -1.f : 1.f;
                sc[i] = ng ? 8388608.f : -8388608.f;
            }
            auto store_slice = [&](auto S_tag) {
                constexpr int S = decltype(S_tag)::value;
                uint32_t w[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    w[q] = oz_pack2(oz_slice<S>(xh[2 * q], xl[2 * q]), sg[2 * q], sc[2 * q],
                                    oz_slice<S>(xh[2 * q + 1], xl[2 * q + 1]), sg[2 * q + 1], sc[2 * q + 1]);
                unsigned char* base = sa + S * kOzSliceA;
                *reinterpret_cast<uint4*>(base + oz_off(r, 16 * half)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(base + oz_off(r, 16 * half + 8)) = make_uint4(w[4], w[5], w[6], w[7]);
            };
            store_slice(std::integral_constant<int, 0>{});
            store_slice(std::integral_constant<int, 1>{});
            store_slice(std::integral_constant<int, 2>{});
            store_slice(std::integral_constant<int, 3>{});
            store_slice(std::integral_constant<int, 4>{});
            store_slice(std::integral_constant<int, 5>{});
            store_slice(std::integral_constant<int, 6>{});
            store_slice(std::integral_constant<int, 7>{});
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(use & 1))) {
                    ok = false;
                } else {
                    tc_fence_after();
                    const uint32_t abase = smem_u32(sa), bbase = smem_u32(sb);
#pragma unroll
                    for (int L = 2; L <= kOzSlices + 1; ++L) {
                        const uint32_t td = tmem + (uint32_t)((L - 2) * kOzNT);
#pragma unroll
                        for (int si = 1; si < L; ++si) {
                            const int sj = L - si;
#pragma unroll
                            for (int kk = 0; kk < kOzKC / 16; ++kk) {
                                const uint64_t ad = make_desc(abase + (si - 1) * kOzSliceA + kk * 256, 128, 512);
                                const uint64_t bd = make_desc(bbase + (sj - 1) * kOzSliceB + kk * 256, 128, 512);
                                mma_bf16(td, ad, bd, idesc, (c > 0 || si > 1 || kk > 0) ? 1u : 0u);
                            }
                        }
                    }
                }
                mma_commit(smem_u32(&done[s]));
                ++committed;
            }
            if (!__syncthreads_and(ok ? 1 : 0)) ok = false;
            if (!ok) break;
        }
        if (!ok) break;
        // epilogue: the item's last products, then TMEM -> FP64
        {
            const int gl = g - 1;
            if (!mbar_wait(smem_u32(&done[gl & 1]), (uint32_t)((gl >> 1) & 1))) ok = false;
        }
        if (!__syncthreads_and(ok ? 1 : 0)) {
            ok = false;
            break;
        }
        tc_fence_after();
        const int q = warp & 3, hc = warp >> 2;
        const int er = q * 32 + lane;  // this thread's TMEM lane = tile row
        const int grow = row0 + er;
        const int erow = max(s_e[er], s_e[kOzTileM + er]);
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hc * 32);
#pragma unroll 1
        for (int cg = 0; cg < 4; ++cg) {
            const int col0 = hc * 32 + cg * 8;  // column within the tile
            if (col0 >= nvalid) break;          // warp-uniform
            uint32_t raw[kOzLevels][8];
#pragma unroll
            for (int l = 0; l < kOzLevels; ++l) tmem_ld8_nowait(tbase + (uint32_t)(l * kOzNT + cg * 8), raw[l]);
            tmem_wait_ld();
            if (grow < a.R) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int col = col0 + j;
                    if (col >= nvalid) continue;
                    const int o = nt * kOzNT + col;
                    float v[kOzLevels];
#pragma unroll
                    for (int l = 0; l < kOzLevels; ++l) v[l] = __uint_as_float(raw[l][j]);
                    double d = oz_combine(v, erow + __ldg(a.B.fexp + o));
                    const size_t oi = (size_t)o * a.R + grow;
                    if (a.dinv) d *= __ldg(a.dinv + oi);
                    a.Out[oi] = d;
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    // drain: products and copies in flight must land before TMEM and shared memory go away
    if (tid == 0) {
        if (committed > 0) {
            const int gl = committed - 1;
            mbar_wait(smem_u32(&done[gl & 1]), (uint32_t)((gl >> 1) & 1));
        }
        for (int q2 = committed; q2 < issued; ++q2) mbar_wait(smem_u32(&full[q2 & 1]), (uint32_t)((q2 >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols));
    }
}

// dinv[k][j n1 + i] = 1 / (lam1[i] + lam2[j] + lam3[k])
__global__ void k_oz_dinv(const double* __restrict__ l1, const double* __restrict__ l2, const double* __restrict__ l3,
                          int n1, int n2, int n3, double* __restrict__ dinv) {
    const size_t N = (size_t)n1 * n2 * n3;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (size_t)gridDim.x * blockDim.x) {
        const size_t k = e / ((size_t)n1 * n2), rem = e - k * (size_t)n1 * n2;
        const int j = (int)(rem / n1), i = (int)(rem - (size_t)j * n1);
        dinv[e] = 1.0 / (l1[i] + l2[j] + l3[k]);
    }
}

int g_oz_sms = 0;

// Host slicing of one mode matrix (row-major n x n, row o = output o).
void slice_matrix(const double* Bm, int n, std::vector<uint16_t>& sl, std::vector<int>& fexp, int& n_tiles,
                  int& k_chunks) {
    n_tiles = (n + kOzNT - 1) / kOzNT;
    k_chunks = (n + kOzKC - 1) / kOzKC;
    const size_t block = (size_t)kOzSlices * kOzNT * kOzKC;  // BF16 values per (tile, chunk)
    sl.assign((size_t)n_tiles * k_chunks * block, 0);
    fexp.assign((size_t)n_tiles * kOzNT, 0);
    for (int o = 0; o < n; ++o) {
        int e = 0;
        for (int t = 0; t < n; ++t) {
            uint64_t b;
            std::memcpy(&b, &Bm[(size_t)o * n + t], 8);
            e = std::max(e, (int)((b >> 52) & 0x7FF));
        }
        fexp[o] = e;
        const int nt = o / kOzNT, rr = o % kOzNT;
        for (int t = 0; t < n; ++t) {
            uint64_t b;
            std::memcpy(&b, &Bm[(size_t)o * n + t], 8);
            const uint64_t X = oz_fixed(b, e);
            const bool neg = (b >> 63) != 0;
            const int kc = t / kOzKC, kk = t % kOzKC;
            uint16_t* blk = sl.data() + ((size_t)nt * k_chunks + kc) * block;
            for (int s = 0; s < kOzSlices; ++s) {
                const int v = (int)((X >> (kOzFix - kOzBits * (s + 1))) & 127u);
                const float f = neg ? -(float)v : (float)v;
                uint32_t fb;
                std::memcpy(&fb, &f, 4);
                blk[((size_t)s * kOzNT * kOzKC * 2 + oz_off(rr, kk)) / 2] = (uint16_t)(fb >> 16);
            }
        }
    }
}

}  // namespace

int configure_fd_oz() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MFWQ_ECUDA;
    if (cudaDeviceGetAttribute(&g_oz_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MFWQ_ECUDA;
    if (cudaFuncSetAttribute(k_fd_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem) != cudaSuccess)
        return MFWQ_ECUDA;
    return MFWQ_OK;
}

int oz_update_dinv(const DirD<double> d64[3], OzPlan& plan, cudaStream_t s) {
    if (!plan.dinv) return MFWQ_EINVAL;
    launch_begin(S_SETUP, s);
    k_oz_dinv<<<1024, 256, 0, s>>>(d64[0].lam, d64[1].lam, d64[2].lam, d64[0].n, d64[1].n, d64[2].n, plan.dinv);
    launch_end(S_SETUP, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}

int oz_plan_build(const Dir1D dir[3], const DirD<double> d64[3], cudaStream_t s, OzPlan& plan) {
    oz_plan_free(plan);
    for (int l = 0; l < 3; ++l)
        if (dir[l].n > kOzMaxN || dir[l].n < 1) return MFWQ_EINVAL;
    std::vector<uint16_t> sl[6];
    std::vector<int> fx[6];
    int nt[6], kc[6];
    for (int l = 0; l < 3; ++l) {
        slice_matrix(dir[l].UT.data(), dir[l].n, sl[l], fx[l], nt[l], kc[l]);          // forward: Bm = U^T
        slice_matrix(dir[l].U.data(), dir[l].n, sl[3 + l], fx[3 + l], nt[3 + l], kc[3 + l]);  // backward: Bm = U
    }
    size_t bytes = 0, off_sl[6], off_fx[6];
    for (int m = 0; m < 6; ++m) {
        off_sl[m] = bytes;
        bytes += (sl[m].size() * 2 + 255) / 256 * 256;
        off_fx[m] = bytes;
        bytes += (fx[m].size() * 4 + 255) / 256 * 256;
    }
    const size_t N = (size_t)dir[0].n * dir[1].n * dir[2].n;
    if (cudaMalloc(&plan.dmem, bytes) != cudaSuccess) return MFWQ_ENOMEM;
    if (cudaMalloc((void**)&plan.dinv, sizeof(double) * N) != cudaSuccess) {
        oz_plan_free(plan);
        return MFWQ_ENOMEM;
    }
    unsigned char* base = static_cast<unsigned char*>(plan.dmem);
    for (int m = 0; m < 6; ++m) {
        if (cudaMemcpy(base + off_sl[m], sl[m].data(), sl[m].size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(base + off_fx[m], fx[m].data(), fx[m].size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            oz_plan_free(plan);
            return MFWQ_ECUDA;
        }
        OzMat& M = m < 3 ? plan.fwd[m] : plan.bwd[m - 3];
        M.sl = reinterpret_cast<const uint16_t*>(base + off_sl[m]);
        M.fexp = reinterpret_cast<const int*>(base + off_fx[m]);
        M.n_out = M.n_in = dir[m % 3].n;
        M.n_tiles = nt[m];
        M.k_chunks = kc[m];
    }
    const int st = oz_update_dinv(d64, plan, s);
    if (st != MFWQ_OK) {
        oz_plan_free(plan);
        return st;
    }
    plan.ok = 1;
    return MFWQ_OK;
}

void oz_plan_free(OzPlan& plan) {
    if (plan.dmem) cudaFree(plan.dmem);
    if (plan.dinv) cudaFree(plan.dinv);
    plan = OzPlan{};
}

namespace {
int oz_pass(const OzMat& B, const double* A, double* Out, int R, const double* dinv, int* err, const int* skip,
            cudaStream_t s) {
    OzArgs a;
    a.A = A;
    a.Out = Out;
    a.B = B;
    a.dinv = dinv;
    a.R = R;
    a.err = err;
    a.skip = skip;
    if (g_rec) {  // no grouped form: a batch with this path runs its patches on streams
        g_rec->unsupported = true;
        return MFWQ_OK;
    }
    const int items = (R + kOzTileM - 1) / kOzTileM * B.n_tiles;
    int grid = g_oz_sms > 0 ? g_oz_sms : 148;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    launch_begin(S_FD_OZ, s);
    k_fd_oz<<<grid, kOzThreads, kOzSmem, s>>>(a);
    launch_end(S_FD_OZ, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}
}  // namespace

int run_fd_oz(const OzPlan& p, const double* r, double* z, double* tmp, int* err, const int* skip, cudaStream_t s) {
    if (!p.ok) return MFWQ_EINVAL;
    const int n1 = p.fwd[0].n_in, n2 = p.fwd[1].n_in, n3 = p.fwd[2].n_in;
    // forward U^T products with the scaling in the third, then the U products (fd_tc.cu's rotation order)
    if (oz_pass(p.fwd[0], r, tmp, n3 * n2, nullptr, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p.fwd[1], tmp, z, n1 * n3, nullptr, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p.fwd[2], z, tmp, n2 * n1, p.dinv, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p.bwd[0], tmp, z, n3 * n2, nullptr, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p.bwd[1], z, tmp, n1 * n3, nullptr, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p.bwd[2], tmp, z, n2 * n1, nullptr, err, skip, s)) return MFWQ_ECUDA;
    return MFWQ_OK;
}

}  // namespace mfwq
