// Tensor-memory-accelerator (TMA) tile loads for sm_103a: tensor maps are
// encoded on the host; a kernel's elected thread issues one
// cp.async.bulk.tensor per tile into shared memory and every thread waits
// on an mbarrier.  Waits are bounded: a wait that runs out sets the batch's
// error word (mapped host memory the runtime checks after every batch) and
// the block returns instead of spinning on.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace flowroi {

constexpr uint32_t kErrTmaTimeout = 1u;  // error word value: a TMA wait ran out
constexpr uint32_t kTmaSpinLimit = 1u << 22;

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes the mbarrier initialisation visible to the async proxy.
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier generic-proxy shared-memory accesses (made
// visible to it by a barrier) before later async-proxy (TMA) writes.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tensormap_acquire(const void *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 3-D tiled load; c0 (innermost) must address a 16-byte boundary.
__device__ __forceinline__ void tma_load_3d(void *dst, const void *map, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Plain arrival (count 1) on an mbarrier.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Barrier over `nthreads` threads only (named barrier `id`, a multiple of
// 32 threads), and the same barrier with an OR reduction of a predicate.
__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ bool named_sync_or(int id, int nthreads, bool p)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, %2, %3, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Bounded wait (at most `limit` polls) for phase `parity` of the mbarrier;
// true when it completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; i++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
#endif

// Host: encode a tiled tensor map (cuTensorMapEncodeTiled through the
// runtime's driver entry point).  dims/strides in elements / bytes as the
// driver API defines them; elements outside dims read as zero.
bool tma_available();
bool tma_encode(CUtensorMap *map, bool half, int rank, void *base, const uint64_t *dims, const uint64_t *strides_bytes,
                const uint32_t *box);

}  // namespace flowroi
