// FD preconditioner mode products on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM), TF32 or BF16 inputs with FP32
// accumulation.  P^-1 r = (U3 (x) U2 (x) U1) diag(1/(l1+l2+l3)) (U3 (x) U2 (x) U1)^T r
// (the FD method of Section 4) as six GEMMs.
//
// Each pass contracts the fastest dimension of its input and writes the new
// index as the slowest dimension of its output ("rotation"):
//     D[r][o] = sum_t A[r][t] Bm[o][t],   Out[o][r] = D[r][o]
// A: input viewed as R rows of n_in contiguous elements; Bm: n_out x n_in
// matrix, K-major.  Three rotations bring the layout back, so
//   x[k][j][i] -U1^T-> [i'][k][j] -U2^T-> [j'][i'][k] -U3^T, /lambda-> [k'][j'][i']
//              -U1-->  [i][k'][j'] -U2--> [j][i][k']  -U3-->  [k][j][i].
// The epilogue store is coalesced: a thread owns a row r (a TMEM lane) and
// consecutive rows are consecutive output addresses.
//
// One CTA = one warpgroup (128 threads) and 128 rows per tile; operands are
// staged through shared memory in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices, LBO = 128 B between K-neighbours, SBO =
// 1024 B between 8-row groups), K chunks of 128 bytes, two stages so that
// the loads of chunk c+1 overlap the MMAs of chunk c.  Every wait on an
// mbarrier is bounded; on timeout the kernel records an error and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "kernels.h"
#include "prof.h"
#include "ptx_async.cuh"

namespace mfwq {
namespace {

using ptx::mbar_expect_tx;
using ptx::mbar_init;
using ptx::mbar_wait;
using ptx::smem_u32;

constexpr int kTcThreads = 128;
constexpr int kTileM = 128;
constexpr int kChunkBytes = 128;           // K bytes per chunk and row
constexpr int kStages = 2;

// Shared-memory matrix descriptor, no swizzle, K-major.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: D = F32, A/B format fmt (TF32 = 2 for kind::tf32,
// BF16 = 1 for kind::f16), both K-major, N and M encoded.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, int M, int N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    if (KIND == 0) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    const float* A;      // [R][n_in]
    const float* Bm;     // [n_out][n_in] (FP32; converted while staging)
    float* Out;          // [n_out][R]
    int R, n_in, n_out, n_pad;  // n_pad: n_out rounded up to 16
    int tmem_cols;
    // scaling epilogue (forward pass along dimension 3): Out /= l1[i] + l2[j] + l3[o], r = j n1 + i
    const float* l1;
    const float* l2;
    const float* l3;
    int n1;
    int* err;
    const int* skip;
};

// Stage one K chunk (kc) of rows [row0, row0 + rows) of a row-major matrix
// src[nrows][ncols] into the canonical layout at dst (row-major core
// matrices: byte (r/8)*1024 + (kb/16)*128 + (r%8)*16 + kb%16).  A warp covers
// 4 rows x 8 consecutive elements per step; each thread issues its loads 16
// at a time into registers before storing them, so the loads are in flight
// together instead of one load-store pair after another.
template <int KIND>
__device__ __forceinline__ void stage_chunk(unsigned char* dst, const float* __restrict__ src, int nrows, int ncols,
                                            int row0, int rows, int kc) {
    constexpr int EB = KIND == 0 ? 4 : 2;  // operand bytes
    constexpr int KE = kChunkBytes / EB;   // elements per chunk row
    constexpr int GROUPS = KE / 8;         // 8-element groups per row
    constexpr int BATCH = 16;
    const int tid = threadIdx.x;
    const int per_thread = rows * KE / kTcThreads;  // rows is a multiple of 16
    for (int base = 0; base < per_thread; base += BATCH) {
        float v[BATCH];
        int off[BATCH];
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            const int idx = base + j;
            v[j] = 0.f;
            off[j] = -1;
            if (idx < per_thread) {
                const int e = tid + idx * kTcThreads;
                const int warp_e = e >> 5, lane = e & 31;
                const int rg = warp_e / GROUPS, kg = warp_e - rg * GROUPS;
                const int r = rg * 4 + (lane >> 3);
                const int k = kg * 8 + (lane & 7);
                const int gr = row0 + r, gk = kc * KE + k;
                if (gr < nrows && gk < ncols) v[j] = src[(size_t)gr * ncols + gk];
                const int kb = k * EB;
                off[j] = (r >> 3) * 1024 + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15);
            }
        }
#pragma unroll
        for (int j = 0; j < BATCH; ++j) {
            if (off[j] < 0) continue;
            if (KIND == 0) {
                *reinterpret_cast<float*>(dst + off[j]) = v[j];
            } else {
                *reinterpret_cast<__nv_bfloat16*>(dst + off[j]) = __float2bfloat16_rn(v[j]);
            }
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(kTcThreads, 1) k_fd_tc(TcArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    // layout: [stages][A 128 rows x 128 B][B n_pad rows x 128 B], then mbarriers and the TMEM address
    const int a_bytes = kTileM * kChunkBytes;
    const int b_bytes = a.n_pad * kChunkBytes;
    const int stage_bytes = a_bytes + b_bytes;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kStages * stage_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + kStages);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&mbar[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    constexpr int EB = KIND == 0 ? 4 : 2;
    constexpr int KE = kChunkBytes / EB;
    constexpr uint32_t FMT = KIND == 0 ? 2u : 1u;
    const uint32_t idesc = make_idesc(FMT, kTileM, a.n_pad);
    const int nchunks = (a.n_in + KE - 1) / KE;
    const int ntiles = (a.R + kTileM - 1) / kTileM;
    bool ok = true;
    int g = 0;  // global chunk counter of this CTA
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int row0 = tile * kTileM;
        for (int c = 0; c < nchunks; ++c, ++g) {
            const int s = g & 1, j = g >> 1;
            unsigned char* sa = smem + s * stage_bytes;
            unsigned char* sb = sa + a_bytes;
            if (j >= 1 && !mbar_wait(smem_u32(&mbar[s]), (uint32_t)((j - 1) & 1))) {
                ok = false;
                break;
            }
            stage_chunk<KIND>(sa, a.A, a.R, a.n_in, row0, kTileM, c);
            stage_chunk<KIND>(sb, a.Bm, a.n_out, a.n_in, 0, a.n_pad, c);
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t abase = smem_u32(sa), bbase = smem_u32(sb);
#pragma unroll
                for (int kk = 0; kk < kChunkBytes / 32; ++kk) {
                    const uint64_t ad = make_desc(abase + kk * 256, 128, 1024);
                    const uint64_t bd = make_desc(bbase + kk * 256, 128, 1024);
                    mma<KIND>(tmem, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(smem_u32(&mbar[s]));
            }
        }
        if (!ok) break;
        // epilogue: wait for the tile's last commit
        const int gl = g - 1;
        if (!mbar_wait(smem_u32(&mbar[gl & 1]), (uint32_t)((gl >> 1) & 1))) {
            ok = false;
            break;
        }
        tc_fence_after();
        const int r = row0 + warp * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
        float inv_ij = 0.f;
        if (a.l3 && r < a.R) {
            const int jj = r / a.n1, ii = r - jj * a.n1;
            inv_ij = a.l1[ii] + a.l2[jj];
        }
        for (int c0 = 0; c0 < a.n_pad; c0 += 16) {
            float v[16];
            tmem_ld16(tbase + c0, v);
            if (r < a.R) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int o = c0 + q;
                    if (o < a.n_out) {
                        float val = v[q];
                        if (a.l3) val = val / (inv_ij + a.l3[o]);
                        a.Out[(size_t)o * a.R + r] = val;
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    // drain: the last commit of this CTA must have completed before TMEM is freed
    if (g > 0) {
        const int gl = g - 1;
        mbar_wait(smem_u32(&mbar[gl & 1]), (uint32_t)((gl >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
    }
}

// ---------------------------------------------------------------- TMA variant (TF32)
// Operands arrive by cp.async.bulk.tensor (2D tiles of 32 FP32 x rows, 128-byte
// swizzle) straight into the canonical SWIZZLE_128B K-major layout the MMA
// reads (8-row x 128-byte atoms, SBO = 1024 B; the K step inside an atom moves
// the descriptor start by 32 B).  One thread issues the copies and the MMAs;
// "full" mbarriers count the copied bytes, "empty" ones are signalled by the
// MMA commit that consumed a stage.  Row strides must be multiples of 16 bytes
// (n_in % 4 == 0); coordinates start at multiples of 32 elements.
constexpr int kTmaStages = 2;

__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: 8-row atoms
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // layout: 128-byte swizzle
    return d;
}


__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

struct TmaArgs {
    float* Out;
    int R, n_in, n_out, n_pad, tmem_cols;
    const float* l1;
    const float* l2;
    const float* l3;
    int n1;
    int* err;
    const int* skip;
};

__global__ void __launch_bounds__(kTcThreads, 1) k_fd_tc_tma(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB, TmaArgs a) {
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned stages: [A 128 x 128 B][B n_pad x 128 B]
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int a_bytes = kTileM * kChunkBytes;
    const int b_bytes = a.n_pad * kChunkBytes;
    const int stage_bytes = a_bytes + b_bytes;  // multiple of 1024 (n_pad is a multiple of 16 -> 2048 B)
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kTmaStages * stage_bytes);
    uint64_t* empty = full + kTmaStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(empty + kTmaStages);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kTmaStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = make_idesc(2u, kTileM, a.n_pad);
    const int nchunks = (a.n_in + 31) / 32;
    const int ntiles = (a.R + kTileM - 1) / kTileM;
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int total = my_tiles * nchunks;  // chunks this CTA consumes, in order
    bool ok = true;
    // producer state (thread 0): next chunk to load
    int loaded = 0;
    auto issue = [&](int g) -> bool {  // load chunk g into stage g % S (thread 0)
        const int s = g % kTmaStages, j = g / kTmaStages;
        if (j >= 1 && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((j - 1) & 1))) return false;
        const int tile = blockIdx.x + (g / nchunks) * gridDim.x;
        const int c = g % nchunks;
        unsigned char* sa = smem + s * stage_bytes;
        mbar_expect_tx(smem_u32(&full[s]), (uint32_t)stage_bytes);
        tma_load_2d(smem_u32(sa), &mapA, c * 32, tile * kTileM, smem_u32(&full[s]));
        tma_load_2d(smem_u32(sa + a_bytes), &mapB, c * 32, 0, smem_u32(&full[s]));
        return true;
    };
    if (tid == 0)
        for (; loaded < total && loaded < kTmaStages; ++loaded) ok = ok && issue(loaded);
    int g = 0;
    for (int ti = 0; ti < my_tiles; ++ti) {
        const int tile = blockIdx.x + ti * gridDim.x;
        const int row0 = tile * kTileM;
        if (tid == 0 && ok) {
            for (int c = 0; c < nchunks; ++c, ++g) {
                const int s = g % kTmaStages, j = g / kTmaStages;
                if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(j & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t abase = smem_u32(smem + s * stage_bytes);
                const uint32_t bbase = abase + a_bytes;
#pragma unroll
                for (int kk = 0; kk < kChunkBytes / 32; ++kk)
                    mma<0>(tmem, make_desc_sw128(abase + kk * 32), make_desc_sw128(bbase + kk * 32), idesc,
                           (c > 0 || kk > 0) ? 1u : 0u);
                mma_commit(smem_u32(&empty[s]));
                if (loaded < total) {
                    if (!issue(loaded)) {
                        ok = false;
                        break;
                    }
                    ++loaded;
                }
            }
        }
        // everyone: wait for the tile's last commit, then read TMEM
        const int gl = (ti + 1) * nchunks - 1;
        __syncthreads();
        if (!mbar_wait(smem_u32(&empty[gl % kTmaStages]), (uint32_t)((gl / kTmaStages) & 1))) ok = false;
        if (!__syncthreads_and(ok ? 1 : 0)) {
            ok = false;
            break;
        }
        tc_fence_after();
        const int r = row0 + warp * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
        float sum_ij = 0.f;
        if (a.l3 && r < a.R) {
            const int jj = r / a.n1, ii = r - jj * a.n1;
            sum_ij = a.l1[ii] + a.l2[jj];
        }
        for (int c0 = 0; c0 < a.n_pad; c0 += 16) {
            float v[16];
            tmem_ld16(tbase + c0, v);
            if (r < a.R) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int o = c0 + q;
                    if (o < a.n_out) {
                        float val = v[q];
                        if (a.l3) val = val / (sum_ij + a.l3[o]);
                        a.Out[(size_t)o * a.R + r] = val;
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    // loads issued but never consumed (only after a failure) and the last commit must land before exit
    if (tid == 0 && total > 0) {
        const int gl = total - 1;
        mbar_wait(smem_u32(&empty[gl % kTmaStages]), (uint32_t)((gl / kTmaStages) & 1));
        for (int q = g; q < loaded; ++q) mbar_wait(smem_u32(&full[q % kTmaStages]), (uint32_t)((q / kTmaStages) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
    }
}

// The tensor-map encoder is a driver entry point; it is looked up through the
// runtime so that the library does not link libcuda directly.
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

bool encode_map(CUtensorMap* m, const float* base, int cols, int rows, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(float)};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int tma_smem_bytes(int n_pad) {
    int b = kTmaStages * (kTileM * kChunkBytes + n_pad * kChunkBytes) + 1024 + 64;  // + alignment slack, barriers
    if (n_pad > 128 && b < 80 * 1024) b = 80 * 1024;
    return b;
}

int g_num_sms = 0;

// Dynamic shared memory of one CTA.  With 256 TMEM columns per CTA at most two
// CTAs may share an SM (512 columns), so the request is raised above a third
// of the SM's shared memory.
int tc_smem_bytes(int n_pad) {
    int b = kStages * (kTileM * kChunkBytes + n_pad * kChunkBytes) + 64;
    if (n_pad > 128 && b < 80 * 1024) b = 80 * 1024;
    return b;
}

template <int KIND>
int launch_pass(const float* A, const float* Bm, float* Out, int R, int n_in, int n_out, const float* l1, const float* l2,
                const float* l3, int n1, int* err, const int* skip, cudaStream_t s) {
    TcArgs a;
    a.skip = skip;
    a.A = A;
    a.Bm = Bm;
    a.Out = Out;
    a.R = R;
    a.n_in = n_in;
    a.n_out = n_out;
    a.n_pad = (n_out + 15) / 16 * 16;
    a.tmem_cols = a.n_pad <= 32 ? 32 : a.n_pad <= 64 ? 64 : a.n_pad <= 128 ? 128 : 256;
    a.l1 = l1;
    a.l2 = l2;
    a.l3 = l3;
    a.n1 = n1;
    a.err = err;
    const int ntiles = (R + kTileM - 1) / kTileM;
    int grid = 2 * g_num_sms;
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    if (KIND == 0 && n_in % 4 == 0 && ((uintptr_t)A & 15) == 0 && ((uintptr_t)Bm & 15) == 0) {
        CUtensorMap ma, mb;
        if (encode_map(&ma, A, n_in, R, kTileM) && encode_map(&mb, Bm, n_in, n_out, a.n_pad)) {
            TmaArgs t;
            t.Out = Out;
            t.R = R;
            t.n_in = n_in;
            t.n_out = n_out;
            t.n_pad = a.n_pad;
            t.tmem_cols = a.tmem_cols;
            t.l1 = l1;
            t.l2 = l2;
            t.l3 = l3;
            t.n1 = n1;
            t.err = err;
            t.skip = skip;
            launch_begin(S_FD_TC, s);
            k_fd_tc_tma<<<grid, kTcThreads, tma_smem_bytes(a.n_pad), s>>>(ma, mb, t);
            launch_end(S_FD_TC, s);
            return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
        }
    }
    launch_begin(S_FD_TC, s);
    k_fd_tc<KIND><<<grid, kTcThreads, tc_smem_bytes(a.n_pad), s>>>(a);
    launch_end(S_FD_TC, s);
    return cudaGetLastError() == cudaSuccess ? MFWQ_OK : MFWQ_ECUDA;
}

template <int KIND>
int run_fd_tc_impl(const DirD<float> d[3], const float* r, float* z, float* tmp, int* err, const int* sk, cudaStream_t s) {
    const int n1 = d[0].n, n2 = d[1].n, n3 = d[2].n;
    // forward: Bm = U^T (row o = column o of U), stored as UT
    if (launch_pass<KIND>(r, d[0].UT, tmp, n3 * n2, n1, n1, nullptr, nullptr, nullptr, 1, err, sk, s)) return MFWQ_ECUDA;
    if (launch_pass<KIND>(tmp, d[1].UT, z, n1 * n3, n2, n2, nullptr, nullptr, nullptr, 1, err, sk, s)) return MFWQ_ECUDA;
    if (launch_pass<KIND>(z, d[2].UT, tmp, n2 * n1, n3, n3, d[0].lam, d[1].lam, d[2].lam, n1, err, sk, s)) return MFWQ_ECUDA;
    // backward: Bm = U
    if (launch_pass<KIND>(tmp, d[0].U, z, n3 * n2, n1, n1, nullptr, nullptr, nullptr, 1, err, sk, s)) return MFWQ_ECUDA;
    if (launch_pass<KIND>(z, d[1].U, tmp, n1 * n3, n2, n2, nullptr, nullptr, nullptr, 1, err, sk, s)) return MFWQ_ECUDA;
    if (launch_pass<KIND>(tmp, d[2].U, z, n2 * n1, n3, n3, nullptr, nullptr, nullptr, 1, err, sk, s)) return MFWQ_ECUDA;
    return MFWQ_OK;
}

}  // namespace

int configure_fd_tc(int max_n) {
    if (max_n > 256) return MFWQ_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MFWQ_ECUDA;
    if (cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MFWQ_ECUDA;
    const int bytes = tc_smem_bytes(256);
    if (cudaFuncSetAttribute(k_fd_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return MFWQ_ECUDA;
    if (cudaFuncSetAttribute(k_fd_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return MFWQ_ECUDA;
    if (cudaFuncSetAttribute(k_fd_tc_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, tma_smem_bytes(256)) != cudaSuccess)
        return MFWQ_ECUDA;
    return MFWQ_OK;
}

int run_fd_tc(const DirD<float> d[3], int fd_precision, const float* r, float* z, float* tmp, int* err, const int* skip,
              cudaStream_t s) {
    if (fd_precision == MFWQ_FD_BF16) return run_fd_tc_impl<1>(d, r, z, tmp, err, skip, s);
    return run_fd_tc_impl<0>(d, r, z, tmp, err, skip, s);
}

}  // namespace mfwq
