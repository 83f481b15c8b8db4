// cluster.cuh -- thread-block cluster primitives for sm_103a kernels: the
// split cluster barrier and distributed shared memory access (PTX ISA:
// barrier.cluster, mapa, ld/st.shared::cluster).
#pragma once
#include <stdint.h>

namespace fcirc {

__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
// Arrive without release semantics: for a thread whose only accesses the
// peers wait on are distributed shared-memory loads whose values it has
// already consumed (a load that fed a later instruction has completed).  It
// does not wait for the thread's outstanding global stores, which the
// release form does.
__device__ __forceinline__ void cl_arrive_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }
__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
// address of the same shared-memory word in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ uint4 cl_ld4(uint32_t a)
{
    uint4 v;
    asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a));
    return v;
}

__device__ __forceinline__ void cl_st4(uint32_t a, uint4 v)
{
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};\n"
                 :
                 : "r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

}  // namespace fcirc
