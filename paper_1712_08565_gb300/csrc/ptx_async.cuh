// Inline-PTX helpers for asynchronous copies into shared memory on sm_103a:
// mbarriers with bounded waits and the 1D bulk copy (cp.async.bulk) that the
// TMA engine executes, completing on an mbarrier's transaction count.
#pragma once

#include <cstdint>

namespace mfwq {
namespace ptx {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: the bound of every wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}

// Makes an initialised mbarrier visible to the async proxy (the copy engine).
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity: false after `limit`
// cycles (kWaitCycles unless a caller asks for less).
__device__ inline bool mbar_wait(uint32_t a, uint32_t parity, long long limit = kWaitCycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(a, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// One arrival that also announces `bytes` of copies completing on the barrier.
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Global -> shared bulk copy of `bytes` (multiple of 16; both addresses
// 16-byte aligned) that completes `bytes` transactions on mbar.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mbar)
                 : "memory");
}

// Per-thread asynchronous global -> shared copy of one 4- or 8-byte element
// (cp.async); completion by cp_async_wait_all in the issuing thread.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async.ca copies 4, 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)),
                 "n"((int)sizeof(T))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Hint to the copy engine: bring [p, p + bytes) into L2 (cp.async.bulk.prefetch.L2);
// p 16-byte aligned, bytes a multiple of 16.  No completion, no effect on results.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p)), "r"(bytes)
                 : "memory");
}

// The same for any byte range: only its 16-byte-aligned interior is prefetched,
// so nothing outside [begin, begin + bytes) is touched; pieces of at most 64 KB.
__device__ inline void prefetch_l2_range(const void* begin, size_t bytes) {
    uint64_t a = (reinterpret_cast<uint64_t>(begin) + 15) & ~uint64_t(15);
    const uint64_t e = (reinterpret_cast<uint64_t>(begin) + bytes) & ~uint64_t(15);
    while (a < e) {
        const uint32_t n = (uint32_t)(e - a < 65536 ? e - a : 65536);
        prefetch_l2(reinterpret_cast<const void*>(a), n);
        a += n;
    }
}

}  // namespace ptx
}  // namespace mfwq
