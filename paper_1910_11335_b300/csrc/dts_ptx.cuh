// dts_ptx.cuh -- inline-PTX wrappers shared by the sweep and the tensor-core
// moment kernel: mbarriers with bounded waits, and bulk-copy TMA
// (cp.async.bulk, no tensor map) between global and shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dts {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// plain arrival (completes a phase without bytes: a copy skipped by a failed bounds check)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: false when the phase did not complete within about a second
// (the caller records an error and stops using the barrier). Each try suspends for at most about
// 20 us; the global timer bounds the total, and an iteration cap bounds it should the timer stall.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    constexpr uint32_t kHintNs = 20000;
    constexpr uint64_t kLimitNs = 1000000000ull;
    constexpr int kMaxTries = 1 << 20;
    if (mbar_try(bar, parity, kHintNs)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (int i = 0; i < kMaxTries; ++i) {
        if (mbar_try(bar, parity, kHintNs)) return true;
        if (globaltimer_ns() - t0 > kLimitNs) return false;
    }
    return false;
}

// global -> shared bulk copy (TMA, no tensor map); bytes and both addresses multiples of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// the mbarrier initialisations of this thread visible to the async proxy (the bulk copies)
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// shared -> global bulk copy (TMA, no tensor map) in this thread's bulk group; bytes and both
// addresses multiples of 16
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// until the shared-memory sources of this thread's committed bulk stores have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// global -> shared tiled copy through a tensor map (TMA, cp.async.bulk.tensor) of a 4-D box at element
// coordinates (c0 innermost; c0 * element size a multiple of 16 bytes); tmap is the generic address
// of a CUtensorMap in kernel-parameter (__grid_constant__), constant or global memory; dst 128-byte
// aligned. Elements outside the tensor arrive as zeros, and the box's full size counts toward bar.
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace dts
