// mbarrier and bulk-copy (TMA, non-tensor) helpers for sm_100-family GPUs.
// Every wait is bounded: it gives up after one second and reports failure,
// so a kernel can flag HERMES_ERR_TIMEOUT instead of hanging the device.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hermes {
namespace ac {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Completion of phase `parity`; false if it did not complete within one second of
// wall time (the global nanosecond timer), or after 2^24 tries, whichever comes first.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (int i = 0; i < (1 << 24); ++i) {
        if (mbar_try(b, parity)) return true;
        if (globaltimer_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}
__device__ __forceinline__ void mbar_inval(uint64_t* b) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(su32(b)) : "memory");
}
// One arrival that also announces `bytes` of transactions (the issuing thread).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// Orders earlier generic-proxy shared-memory accesses before later async-proxy ones.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Bulk copy global -> this CTA's shared memory; both addresses 16-byte aligned,
// bytes a multiple of 16; completion is signalled on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

// Tiled bulk store (TMA) of one 3-D box from this CTA's shared memory to global memory,
// described by a tensor map that is a __grid_constant__ kernel parameter; coordinates in
// elements, the innermost one times the element size a multiple of 16 bytes; the shared
// source 16-byte aligned, its generic-proxy writes ordered before by fence_proxy_async.
// The store joins the calling thread's current bulk group; commit closes the group.
__device__ __forceinline__ void tma_store_3d(const void* tmap, const void* src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(tmap),
                 "r"(su32(src)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Until every committed bulk group of this thread has read its shared source (the copies
// always complete: no bound needed), so the source may be overwritten.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Until every committed bulk group of this thread has completed its global writes.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared (both 16-byte aligned), in the
// calling thread's current group; commit closes the group, wait_all waits for
// every group of this thread (the copies always complete: no bound needed).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace ac
}  // namespace hermes
