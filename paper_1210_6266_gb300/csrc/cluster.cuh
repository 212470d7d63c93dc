// Thread-block cluster primitives (sm_90 and later): the CTA's rank in its cluster, the
// cluster-wide barrier, and loads from a peer CTA's shared memory (distributed shared
// memory, addresses mapped with mapa).
#pragma once
#include <cstdint>

namespace rsd {

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// all threads of every CTA of the cluster (uniform control flow only); release/acquire
// orders each CTA's earlier shared-memory writes before the peers' later reads
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// the shared::cluster address of p (a shared variable of this CTA) in CTA `rank`
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ int cl_ld(uint32_t a) {
    int v;
    asm volatile("ld.shared::cluster.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ double cl_ld_f64(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}

}  // namespace rsd
