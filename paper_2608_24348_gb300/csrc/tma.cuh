// tma.cuh -- bulk asynchronous copies (cp.async.bulk) with mbarrier completion.
//
// Used to stream contiguous per-element-group blocks (a slab of u and the
// element-blocked geometric factors) from HBM into shared memory while the
// block computes on the previous group.  Every wait is bounded in time: a
// wait that runs out reports false and the caller records an error instead
// of spinning forever.
#pragma once

#include <stdint.h>

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the asynchronous proxy.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared accesses before later
// asynchronous-proxy (bulk copy) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// dst (shared) <- src (global), bytes a multiple of 16, both 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long tma_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of bar to complete, at most timeout_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long timeout_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = tma_clock_ns();
    while (!mbar_try_wait(bar, parity)) {
        if ((long long)(tma_clock_ns() - t0) > timeout_ns) return false;
    }
    return true;
}

// Hint: start moving [src, src + bytes) from HBM into L2 (bytes a multiple of
// 16, src 16-byte aligned).  Nothing completes or waits; a later load of the
// same lines finds them in L2.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// L2 prefetch of the bytes [begin, end) of a buffer, shrunk to whole 16-byte
// units inside it, so no prefetched byte lies outside the buffer.
__device__ __forceinline__ void l2_prefetch_span(const void *base, int64_t begin, int64_t end)
{
    const uintptr_t b = ((uintptr_t)base + (uintptr_t)begin + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)base + (uintptr_t)end) & ~(uintptr_t)15;
    if (e > b) bulk_prefetch_l2((const void *)b, (uint32_t)(e - b));
}
