// FP64-accurate FD mode products on the BF16 tensor cores by operand
// splitting (see fd_oz.h for the scheme and its error bound).
//
// One pass contracts the fastest dimension of its input and writes the new
// index as the slowest dimension of its output, as the TF32/BF16 passes of
// fd_tc.cu do:  D[r][o] = sum_t A[r][t] Bm[o][t],  Out[o][r] = D[r][o].
//
// A pass is two kernels.
//  * k_oz_slice (one warp per row of A, coalesced): the row's largest biased
//    exponent, then each element split into its 8 slices with integer
//    operations and stored as BF16 in blocks laid out as the MMA reads them
//    (one block per 128 rows and K chunk), beside the row exponents.
//  * k_fd_oz (512 threads, one CTA per SM: its TMEM blocks take the 512
//    columns) computes 128 rows x kOzNT outputs per work item.  Thread 0
//    streams the slice blocks of A and Bm for each K chunk of 16 elements by
//    bulk copies into four shared-memory stages (three chunks ahead) and
//    issues the 36 slice-pair products of a chunk into the TMEM blocks of
//    their levels, committing to the stage's mbarrier.  Epilogue: warp w
//    reads TMEM lanes 32 (w % 4) .. + 31 and a quarter of the columns; per output the
//    8 level sums (integers in FP32) are converted to integers, added with
//    their weights 2^(7 (9 - L)) in 128 bits and rounded to FP64 by
//    constructing the bit pattern with the row and column scales; the scaling
//    pass multiplies by 1 / (lam1 + lam2 + lam3) from a table.
// Every mbarrier wait is bounded; on timeout the kernel records an error,
// waits (bounded) for its copies and products in flight, frees TMEM and
// returns.
#include <cuda_runtime.h>

#include <algorithm>
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

constexpr int kOzThreads = 512;  // 16 warps: 4 TMEM lane quarters x 4 column quarters in the epilogue
constexpr int kOzTileM = 128;
constexpr int kOzSliceA = kOzTileM * kOzKC * 2;    // bytes of one A slice tile (4 KB)
constexpr int kOzSliceB = kOzNT * kOzKC * 2;       // bytes of one Bm slice tile (2 KB)
constexpr int kOzStageA = kOzSlices * kOzSliceA;   // 32 KB
constexpr int kOzStageB = kOzSlices * kOzSliceB;   // 16 KB
constexpr int kOzStage = kOzStageA + kOzStageB;
constexpr int kOzStages = 4;
constexpr int kOzTmemCols = 512;                   // kOzLevels * kOzNT
constexpr int kOzSmem = kOzStages * kOzStage + 1024 /* alignment */ + 128 /* barriers, TMEM address */;

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

// ---- slicing pre-pass: one warp per (padded) row of A, lane l holds
// elements 8 l .. 8 l + 7 (one 16-byte core-matrix row per slice)
struct OzSliceArgs {
    const double* A;  // [R][n_in]
    int R, n_in, kch, rows_pad;
    uint16_t* sl;     // slice blocks (OzPlan::asl)
    int* aexp;        // row exponents
};

// Block blk of 256 threads: rows 8 blk .. 8 blk + 7.  No early return: the
// grouped launch runs it between block-wide barriers.
__device__ __forceinline__ void oz_slice_body(const OzSliceArgs& a, int blk) {
    const int lane = threadIdx.x & 31;
    const int row = blk * 8 + (int)(threadIdx.x >> 5);
    if (row < a.rows_pad) {
        const int t0 = 8 * lane;
        unsigned long long b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) b[i] = 0ull;
        if (row < a.R && t0 < a.n_in) {
            const double* p = a.A + (size_t)row * a.n_in + t0;
            if (t0 + 8 <= a.n_in && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const double2 v = __ldg(reinterpret_cast<const double2*>(p) + i);
                    b[2 * i] = (unsigned long long)__double_as_longlong(v.x);
                    b[2 * i + 1] = (unsigned long long)__double_as_longlong(v.y);
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (t0 + i < a.n_in) b[i] = (unsigned long long)__double_as_longlong(__ldg(p + i));
            }
        }
        int e = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) e = max(e, (int)((b[i] >> 52) & 0x7FF));
        const int emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
        if (lane == 0) a.aexp[row] = emax;
        if (t0 < a.kch * kOzKC) {  // lanes beyond the padded K write nothing
            uint32_t xh[8], xl[8];
            float sg[8], sc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint64_t X = oz_fixed(b[i], emax);
                xh[i] = (uint32_t)(X >> 32);
                xl[i] = (uint32_t)X;
                const bool ng = (b[i] >> 63) != 0ull;
                sg[i] = ng ? -1.f : 1.f;
                sc[i] = ng ? 8388608.f : -8388608.f;
            }
            const int mt = row / kOzTileM, rr = row - mt * kOzTileM, kc = t0 / kOzKC;
            unsigned char* blkp =
                reinterpret_cast<unsigned char*>(a.sl) + ((size_t)mt * a.kch + kc) * kOzStageA + oz_off(rr, t0 % kOzKC);
            auto put = [&](auto S_tag) {
                constexpr int S = decltype(S_tag)::value;
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    w[q] = oz_pack2(oz_slice<S>(xh[2 * q], xl[2 * q]), sg[2 * q], sc[2 * q],
                                    oz_slice<S>(xh[2 * q + 1], xl[2 * q + 1]), sg[2 * q + 1], sc[2 * q + 1]);
                *reinterpret_cast<uint4*>(blkp + S * kOzSliceA) = make_uint4(w[0], w[1], w[2], w[3]);
            };
            put(std::integral_constant<int, 0>{});
            put(std::integral_constant<int, 1>{});
            put(std::integral_constant<int, 2>{});
            put(std::integral_constant<int, 3>{});
            put(std::integral_constant<int, 4>{});
            put(std::integral_constant<int, 5>{});
            put(std::integral_constant<int, 6>{});
            put(std::integral_constant<int, 7>{});
        }
    }
}

__global__ void __launch_bounds__(256) k_oz_slice(OzSliceArgs a, const int* skip) {
    if (skip && *skip) return;
    oz_slice_body(a, (int)blockIdx.x);
}

// The slicing passes of a batch's patches in one launch (grouped.h).
__global__ void __launch_bounds__(256) k_oz_slice_grouped(const unsigned char* __restrict__ tab, int stride, int npatch) {
    grouped_for<OzSliceArgs, false>(tab, stride, npatch, [](const OzSliceArgs& a, int it) { oz_slice_body(a, it); });
}

struct OzArgs {
    const uint16_t* Asl;  // A slices, [mtiles][k_chunks] blocks of kOzStageA bytes (k_oz_slice)
    const int* aexp;      // [mtiles * 128]: row exponents of A
    double* Out;          // [n_out][R]
    OzMat B;
    const double* dinv;   // null, or the [n_out][R] scaling table
    int R;
    int* err;
    const int* skip;
};

// Epilogue of one work item: warp w reads TMEM lanes 32 (w % 4) .. + 31 and a
// quarter of the tile's columns, combines the 8 level sums of each output into
// FP64 and stores it (times the scaling table in the scaling pass).
__device__ __forceinline__ void oz_epilogue(const OzArgs& a, uint32_t tmem, int row0, int nt, int nvalid) {
    constexpr int kColsPerWarp = kOzNT / (kOzThreads / 128);  // 16
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3, hc = warp >> 2;
    const int er = q * 32 + lane;  // this thread's TMEM lane = tile row
    const int grow = row0 + er;
    const int erow = __ldg(a.aexp + row0 + er);
    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hc * kColsPerWarp);
#pragma unroll 1
    for (int cg = 0; cg < kColsPerWarp / 8; ++cg) {
        const int col0 = hc * kColsPerWarp + cg * 8;  // column within the tile
        if (col0 >= nvalid) break;                     // warp-uniform
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
}

// The slice-pair products of one K chunk (stage at abase / bbase) into the
// TMEM blocks of their levels (thread 0); the first chunk of an item overwrites.
__device__ __forceinline__ void oz_mma_chunk(uint32_t tmem, uint32_t abase, uint32_t bbase, uint32_t idesc, bool first) {
    const uint64_t ad0 = make_desc(abase, 128, kOzSBO), bd0 = make_desc(bbase, 128, kOzSBO);
#pragma unroll
    for (int L = 2; L <= kOzSlices + 1; ++L) {
        const uint32_t td = tmem + (uint32_t)((L - 2) * kOzNT);
#pragma unroll
        for (int si = 1; si < L; ++si) {
#pragma unroll
            for (int kk = 0; kk < kOzKC / 16; ++kk) {
                // descriptor start addresses advance in 16-byte units
                const uint64_t ad = ad0 + (uint64_t)(((si - 1) * kOzSliceA + kk * 256) >> 4);
                const uint64_t bd = bd0 + (uint64_t)(((L - si - 1) * kOzSliceB + kk * 256) >> 4);
                mma_bf16(td, ad, bd, idesc, (!first || si > 1 || kk > 0) ? 1u : 0u);
            }
        }
    }
}

// ---- products: thread 0 streams the slice blocks of A and Bm by bulk copies
// (one chunk ahead) and issues the MMAs; all warps run the epilogue.
__global__ void __launch_bounds__(kOzThreads, 1) k_fd_oz(OzArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOzStages * kOzStage);  // a stage's slices arrived
    uint64_t* done = full + kOzStages;                                          // a stage's products finished
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + kOzStages);
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

    const int n_out = a.B.n_out, kch = a.B.k_chunks, ntl = a.B.n_tiles;
    const int mtiles = (a.R + kOzTileM - 1) / kOzTileM;
    const int items = mtiles * ntl;
    const int my_items = (int)blockIdx.x < items ? (items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = my_items * kch;  // chunks of this CTA, in order
    bool ok = true;
    int issued = 0, committed = 0;  // thread 0: chunk copies started, chunk products committed
    // thread 0: start the copies of chunk q (stage q % kOzStages); the stage's products of chunk q - kOzStages
    // must have finished
    auto issue = [&](int q) -> bool {
        const int s = q % kOzStages, use = q / kOzStages;
        if (use >= 1 && !mbar_wait(smem_u32(&done[s]), (uint32_t)((use - 1) & 1))) return false;
        const int it = (int)blockIdx.x + (q / kch) * (int)gridDim.x, c = q % kch;
        const int mt = it / ntl, nt = it - mt * ntl;
        unsigned char* sa = smem + s * kOzStage;
        mbar_expect_tx(smem_u32(&full[s]), (uint32_t)kOzStage);
        ptx::bulk_g2s(smem_u32(sa), reinterpret_cast<const unsigned char*>(a.Asl) + ((size_t)mt * kch + c) * kOzStageA,
                      (uint32_t)kOzStageA, smem_u32(&full[s]));
        ptx::bulk_g2s(smem_u32(sa + kOzStageA),
                      reinterpret_cast<const unsigned char*>(a.B.sl) + ((size_t)nt * kch + c) * kOzStageB,
                      (uint32_t)kOzStageB, smem_u32(&full[s]));
        ++issued;
        return true;
    };
    if (tid == 0)
        for (int q = 0; q < kOzStages - 1 && q < total && ok; ++q) ok = issue(q);
    int g = 0;
    for (int ii = 0; ii < my_items; ++ii) {
        const int item = (int)blockIdx.x + ii * (int)gridDim.x;
        const int mt = item / ntl, nt = item - mt * ntl;
        const int row0 = mt * kOzTileM;
        const int nvalid = min(kOzNT, n_out - nt * kOzNT);
        if (tid == 0 && ok) {
            const uint32_t idesc = idesc_bf16((nvalid + 15) & ~15);
            for (int c = 0; c < kch; ++c, ++g) {
                const int s = g % kOzStages, use = g / kOzStages;
                if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(use & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t abase = smem_u32(smem + s * kOzStage), bbase = abase + kOzStageA;
                oz_mma_chunk(tmem, abase, bbase, idesc, c == 0);
                mma_commit(smem_u32(&done[s]));
                ++committed;
                if (g + kOzStages - 1 < total && !issue(g + kOzStages - 1)) {
                    ok = false;
                    ++g;
                    break;
                }
            }
            // the item's products complete with its last chunk's commit
            if (ok) {
                const int gl = g - 1;
                if (!mbar_wait(smem_u32(&done[gl % kOzStages]), (uint32_t)((gl / kOzStages) & 1))) ok = false;
            }
        }
        if (!__syncthreads_and(ok ? 1 : 0)) {
            ok = false;
            break;
        }
        tc_fence_after();
        oz_epilogue(a, tmem, row0, nt, nvalid);
        tc_fence_before();
        __syncthreads();  // TMEM is read: the next item's products may overwrite it
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    // drain: products and copies in flight must land before TMEM and shared memory go away
    if (tid == 0) {
        if (committed > 0) {
            const int gl = committed - 1;
            mbar_wait(smem_u32(&done[gl % kOzStages]), (uint32_t)((gl / kOzStages) & 1));
        }
        for (int q2 = committed; q2 < issued; ++q2)
            mbar_wait(smem_u32(&full[q2 % kOzStages]), (uint32_t)((q2 / kOzStages) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols));
    }
}

// The product passes of a batch's patches in one launch (grouped.h): the
// CTAs walk every live patch's work items (table of OzArgs); per item thread 0
// starts its first chunks' copies, consumes the chunks in order with the
// copies of later chunks kept up to three ahead, and all warps run the
// epilogue.  Chunks are counted over the whole launch for the stage barriers.
__global__ void __launch_bounds__(kOzThreads, 1) k_fd_oz_grouped(const unsigned char* __restrict__ tab, int stride,
                                                               int npatch) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOzStages * kOzStage);
    uint64_t* done = full + kOzStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + kOzStages);
    const int tid = threadIdx.x, warp = tid >> 5;
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
    int issued = 0, g = 0, committed = 0;  // thread 0: chunk copies started, consumed, committed
    bool ok = true;
    int* err = nullptr;
    grouped_for<OzArgs, false>(tab, stride, npatch, [&](const OzArgs& a, int item) {
        if (!ok) return;  // uniform: set from a block-wide vote
        err = a.err;
        const int ntl = a.B.n_tiles, kch = a.B.k_chunks;
        const int mt = item / ntl, nt = item - mt * ntl;
        const int row0 = mt * kOzTileM;
        const int nvalid = min(kOzNT, a.B.n_out - nt * kOzNT);
        if (tid == 0) {
            // chunk c of this item into stage issued % kOzStages, once that stage's previous products finished
            auto issue = [&](int c) -> bool {
                const int q = issued, s = q % kOzStages, use = q / kOzStages;
                if (use >= 1 && !mbar_wait(smem_u32(&done[s]), (uint32_t)((use - 1) & 1))) return false;
                unsigned char* sa = smem + s * kOzStage;
                mbar_expect_tx(smem_u32(&full[s]), (uint32_t)kOzStage);
                ptx::bulk_g2s(smem_u32(sa),
                              reinterpret_cast<const unsigned char*>(a.Asl) + ((size_t)mt * kch + c) * kOzStageA,
                              (uint32_t)kOzStageA, smem_u32(&full[s]));
                ptx::bulk_g2s(smem_u32(sa + kOzStageA),
                              reinterpret_cast<const unsigned char*>(a.B.sl) + ((size_t)nt * kch + c) * kOzStageB,
                              (uint32_t)kOzStageB, smem_u32(&full[s]));
                ++issued;
                return true;
            };
            bool lok = true;
            for (int c = 0; c < kOzStages - 1 && c < kch && lok; ++c) lok = issue(c);
            const uint32_t idesc = idesc_bf16((nvalid + 15) & ~15);
            for (int c = 0; c < kch && lok; ++c, ++g) {
                const int s = g % kOzStages, use = g / kOzStages;
                if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(use & 1))) {
                    lok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t abase = smem_u32(smem + s * kOzStage), bbase = abase + kOzStageA;
                oz_mma_chunk(tmem, abase, bbase, idesc, c == 0);
                mma_commit(smem_u32(&done[s]));
                ++committed;
                if (c + kOzStages - 1 < kch && !issue(c + kOzStages - 1)) {
                    lok = false;
                    ++g;
                    break;
                }
            }
            if (lok) {
                const int gl = g - 1;
                if (!mbar_wait(smem_u32(&done[gl % kOzStages]), (uint32_t)((gl / kOzStages) & 1))) lok = false;
            }
            ok = lok;
        }
        if (!__syncthreads_and(ok ? 1 : 0)) {
            ok = false;
            return;
        }
        tc_fence_after();
        oz_epilogue(a, tmem, row0, nt, nvalid);
        tc_fence_before();
        __syncthreads();  // TMEM is read: the next item's products may overwrite it
    });
    if (!ok && tid == 0 && err) atomicExch(err, 1);
    if (tid == 0) {
        if (committed > 0) {
            const int gl = committed - 1;
            mbar_wait(smem_u32(&done[gl % kOzStages]), (uint32_t)((gl / kOzStages) & 1));
        }
        for (int q2 = committed; q2 < issued; ++q2)
            mbar_wait(smem_u32(&full[q2 % kOzStages]), (uint32_t)((q2 / kOzStages) & 1));
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
    if (cudaFuncSetAttribute(k_fd_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_fd_oz_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem) != cudaSuccess)
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
    size_t asl_bytes = 0, aexp_n = 0;
    for (int l = 0; l < 3; ++l) {
        const size_t R = N / dir[l].n, mt = (R + kOzTileM - 1) / kOzTileM;
        asl_bytes = std::max(asl_bytes, mt * (size_t)kc[l] * kOzStageA);
        aexp_n = std::max(aexp_n, mt * kOzTileM);
    }
    if (cudaMalloc(&plan.dmem, bytes) != cudaSuccess) return MFWQ_ENOMEM;
    if (cudaMalloc((void**)&plan.dinv, sizeof(double) * N) != cudaSuccess ||
        cudaMalloc((void**)&plan.asl, asl_bytes) != cudaSuccess ||
        cudaMalloc((void**)&plan.aexp, sizeof(int) * aexp_n) != cudaSuccess) {
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
    if (plan.asl) cudaFree(plan.asl);
    if (plan.aexp) cudaFree(plan.aexp);
    plan = OzPlan{};
}

namespace {
int oz_pass(const OzPlan& p, const OzMat& B, const double* A, double* Out, int R, const double* dinv, int* err,
            const int* skip, cudaStream_t s) {
    OzArgs a;
    a.Asl = p.asl;
    a.aexp = p.aexp;
    a.Out = Out;
    a.B = B;
    a.dinv = dinv;
    a.R = R;
    a.err = err;
    a.skip = skip;
    const int mtiles = (R + kOzTileM - 1) / kOzTileM;
    const int items = mtiles * B.n_tiles;
    const int rows_pad = mtiles * kOzTileM;
    const OzSliceArgs sa{A, R, B.n_in, B.k_chunks, rows_pad, p.asl, p.aexp};
    if (g_rec) {  // the batch's grouped sweep runs both passes over all its patches
        record_launch(GK_OZ_SLICE, sa, (rows_pad + 7) / 8, 256, 0, skip);
        record_launch(GK_OZ_PROD, a, items, kOzThreads, kOzSmem, skip);
        return MFWQ_OK;
    }
    int grid = g_oz_sms > 0 ? g_oz_sms : 148;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    launch_begin(S_FD_OZ, s);
    k_oz_slice<<<(rows_pad + 7) / 8, 256, 0, s>>>(sa, skip);
    launch_end(S_FD_OZ, s);
    launch_begin(S_FD_OZ, s);
    k_fd_oz<<<grid, kOzThreads, kOzSmem, s>>>(a);
    launch_end(S_FD_OZ, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}
}  // namespace

bool grouped_launch_oz(int kind, const unsigned char* tab, int stride, int npatch, int grid, int smem, cudaStream_t s) {
    (void)smem;
    if (kind == GK_OZ_SLICE) {
        k_oz_slice_grouped<<<grid, 256, 0, s>>>(tab, stride, npatch);
        return true;
    }
    if (kind == GK_OZ_PROD) {  // one CTA per SM (shared memory and TMEM)
        const int sms = g_oz_sms > 0 ? g_oz_sms : 148;
        k_fd_oz_grouped<<<grid < sms ? grid : sms, kOzThreads, kOzSmem, s>>>(tab, stride, npatch);
        return true;
    }
    return false;
}

int run_fd_oz(const OzPlan& p, const double* r, double* z, double* tmp, int* err, const int* skip, cudaStream_t s) {
    if (!p.ok) return MFWQ_EINVAL;
    const int n1 = p.fwd[0].n_in, n2 = p.fwd[1].n_in, n3 = p.fwd[2].n_in;
    // forward U^T products with the scaling in the third, then the U products (fd_tc.cu's rotation order)
    if (oz_pass(p, p.fwd[0], r, tmp, n3 * n2, nullptr, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p, p.fwd[1], tmp, z, n1 * n3, nullptr, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p, p.fwd[2], z, tmp, n2 * n1, p.dinv, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p, p.bwd[0], tmp, z, n3 * n2, nullptr, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p, p.bwd[1], z, tmp, n1 * n3, nullptr, err, skip, s)) return MFWQ_ECUDA;
    if (oz_pass(p, p.bwd[2], tmp, z, n2 * n1, nullptr, err, skip, s)) return MFWQ_ECUDA;
    return MFWQ_OK;
}

}  // namespace mfwq
