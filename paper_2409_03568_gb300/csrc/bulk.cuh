// bulk.cuh -- staging of contiguous global-memory segments into shared memory by the tensor
// memory accelerator's bulk copies (cp.async.bulk, completion counted on an mbarrier), with
// bounded waits.
//
// A block keeps S stages of shared memory; one thread issues the bulk copies of a stage and
// announces their byte count on the stage's mbarrier, every thread waits on the barrier's phase
// before reading the stage. Waits are bounded: a wait that gives up returns false, and the
// block's threads agree on it before anyone leaves (no thread is left at a barrier).
#pragma once
#include "common.cuh"

namespace ichee {

// Iterations of mbarrier.try_wait before a wait gives up (each try may suspend the thread for a
// while; this is seconds, far beyond any copy's latency).
constexpr u32 kBulkWaitTries = 1u << 24;

__device__ __forceinline__ u32 smem_addr(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64* bar, u32 arrivals)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(arrivals) : "memory");
}

// Make initialised barriers visible to the bulk-copy engine (call once, before the block's
// first copy; a __syncthreads must follow).
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Order this thread's earlier shared-memory accesses before bulk copies it issues next (the
// stage being refilled was read by the block's threads; a __syncthreads precedes this).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Arrive once on the barrier and add `bytes` to the transaction count of its current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(u64* bar, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to shared
// memory; its completion is counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity)
{
    u32 done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase with the given parity to complete; false if it did not within the bound.
__device__ __forceinline__ bool mbar_wait(u64* bar, u32 parity)
{
    for (u32 i = 0; i < kBulkWaitTries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace ichee
