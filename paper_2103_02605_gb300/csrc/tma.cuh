// tma.cuh -- the tensor memory accelerator (TMA) and shared-memory mbarrier
// operations the kernels use, as inline PTX: tiled tensor copies between
// global and shared memory, completion tracked on an mbarrier (loads) or in
// bulk groups (stores).  Every tensor map covers this GPU's own buffers, and
// no copy uses cluster multicast.
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace fcirc {

__device__ __forceinline__ uint32_t sm_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sm_u32(bar)), "r"(count) : "memory");
    // the initialisation is visible to the async proxy (the TMA unit)
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Arrives on the barrier and adds `bytes` to the transaction count its
// current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sm_u32(bar)), "r"(bytes)
                 : "memory");
}

// One bounded probe: true once the phase with this parity has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(sm_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with at most `limit` probes; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Tiled 4-D load of one box of `map` at coordinates (c0, c1, c2, c3) into
// shared memory at dst (128-byte aligned); completes on `bar` with the box's
// bytes.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(sm_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(sm_u32(bar))
        : "memory");
}

// Tiled 4-D store of one box from shared memory at src into `map` at
// (c0, c1, c2, c3); tracked in the issuing thread's bulk group.
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const void *src, int c0, int c1, int c2, int c3)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];\n" ::"l"(map),
                 "r"(sm_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

// Tiled 5-D store of one box from shared memory at src into `map` at
// (c0, .., c4); tracked in the issuing thread's bulk group.
__device__ __forceinline__ void tma_store_5d(const CUtensorMap *map, const void *src, int c0, int c1, int c2, int c3,
                                             int c4)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5, %6}], [%1];\n" ::"l"(map),
        "r"(sm_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

__device__ __forceinline__ void tma_store_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }

// Waits until the committed stores have read their shared-memory sources
// (the CTA may then leave or reuse that memory).
__device__ __forceinline__ void tma_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }

// Orders this thread's ordinary shared-memory writes before later TMA reads
// of them (issued after a barrier).
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

}  // namespace fcirc
