// Bulk-copy (TMA engine) and mbarrier helpers for sm_103a, as inline PTX.
//
// The tape adjoint reads the forward tape's steps into a shared-memory ring, and the contraction
// streams the dk/dM buffer the same way: cp.async.bulk (shared <- global) completing on per-slot
// mbarriers.  Every wait is bounded; a wait that runs out sets the device error word
// (SK_ERR_DEVICE_TIMEOUT) and reports failure.
#pragma once

#include <stdint.h>

#include "sk_common.cuh"

namespace sk {

constexpr uint32_t kWaitLimit = 1u << 20;  // try_wait polls before a wait is declared stuck

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes the barrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false (and the device error word set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    record_error(SK_ERR_DEVICE_TIMEOUT);
    return false;
}

// Orders this thread's shared-memory accesses in the generic proxy (ordinary loads and stores,
// and those of the threads it synchronised with) before its later async-proxy operations (bulk
// copies, tensor-core reads), and the other way round.  A ring slot that the warp has read must
// be fenced so before a bulk copy refills it: without the fence the copy may land before a
// pending shared-memory load of the slot has read it (seen as corrupted adjoints when another
// kernel's stores kept the load/store units busy).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Per-thread asynchronous copies global -> shared (cp.async, 16 or 8 bytes, both addresses aligned
// to the size), grouped by commit_group; wait_group<N> returns once at most N of the thread's
// groups are still in flight.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

// global -> shared, `bytes` (multiple of 16, both addresses 16-byte aligned), completing on `bar`.
__device__ __forceinline__ void bulk_load(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace sk
