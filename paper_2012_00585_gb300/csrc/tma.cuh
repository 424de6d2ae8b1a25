// Bulk asynchronous copies (TMA, non-tensor form) global -> shared memory,
// completed on an mbarrier, for sm_100-family GPUs.  Every wait is bounded.
#pragma once

#include <stdint.h>

// Spin limit for one mbarrier phase (try_wait may also suspend in hardware
// for a while per call); after it the caller reports FE_ERR_TIMEOUT.
#define FE_MBAR_SPIN_LIMIT (1u << 22)

__device__ __forceinline__ uint32_t fe_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void fe_mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(fe_smem_u32(bar)), "r"(count) : "memory");
}

// Makes mbarrier initialisation visible to the asynchronous proxy.
__device__ __forceinline__ void fe_fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier shared-memory accesses before later
// asynchronous-proxy writes to the same buffer.
__device__ __forceinline__ void fe_fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fe_mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fe_smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t fe_policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void fe_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            fe_smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(fe_smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ bool fe_mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(fe_smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; false on timeout.
__device__ __forceinline__ bool fe_mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < FE_MBAR_SPIN_LIMIT; ++i)
        if (fe_mbar_try_wait(bar, parity)) return true;
    return false;
}
