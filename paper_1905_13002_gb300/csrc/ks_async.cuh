// ks_async.cuh -- bulk asynchronous copies (TMA, cp.async.bulk) between
// global and shared memory, tracked by per-lane mbarriers (loads) and bulk
// groups (stores), with bounded waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifndef KS_DEV
#define KS_DEV __device__ __forceinline__
#endif

namespace ks {

KS_DEV uint32_t smem_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses to the same memory.
KS_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the kernel before it in the stream drains;
// pdl_wait() blocks until that kernel has completed and its memory writes are
// visible (a no-op for a kernel launched without the attribute), and
// pdl_trigger() lets the next such kernel be scheduled once every block of
// this grid has triggered or exited.
KS_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
KS_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Global <- shared bulk copy (bytes % 16 == 0, both addresses 16-byte aligned).
KS_DEV void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 :: "l"(gdst), "r"(smem_addr(ssrc)), "r"(bytes) : "memory");
}
KS_DEV void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until every committed bulk store has finished reading shared memory.
KS_DEV void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Wait until every committed bulk store has completed.
KS_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

KS_DEV void mbar_init(uint64_t* m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(m)), "r"(count) : "memory");
}

// Arrive on `m` announcing `bytes` of incoming transaction data.
KS_DEV void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(m)), "r"(bytes) : "memory");
}

// Shared <- global bulk copy completing on mbarrier `m`.
KS_DEV void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_addr(sdst)), "l"(gsrc), "r"(bytes), "r"(smem_addr(m)) : "memory");
}

KS_DEV bool mbar_try_wait(uint64_t* m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_addr(m)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `m`; false if it never completed.
KS_DEV bool mbar_wait(uint64_t* m, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(m, parity)) return true;
        if (it > 16) __nanosleep(64);
    }
    return false;
}

}  // namespace ks
