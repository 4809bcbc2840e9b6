// Bulk asynchronous copies (the TMA engine's untiled form) into shared
// memory, completed on an mbarrier, and bounded waits on that barrier: a
// wait gives up after a fixed number of polls, latches a status word in
// device memory and lets the kernel return, so a copy that never lands
// cannot hang the GPU. mbc_sync_status reads and clears the word.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace mbc {

// Latched device status of the kernels (per device): bit 0 = a bounded wait
// ran out. Zero when nothing went wrong.
__device__ unsigned int g_device_status;
constexpr unsigned int kStatusWaitTimeout = 1u;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the async proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces tx_bytes of copies to come
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t tx_bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(tx_bytes)
                 : "memory");
}

// bytes (a multiple of 16) from global src to shared dst, both 16-byte
// aligned; counted against bar's transaction count when they land
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy ones (a bulk copy overwriting what was just read)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase with the given parity to complete, polling at most
// limit times; false when the limit ran out (the status word is then set).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        __nanosleep(64);
    }
    atomicOr(&g_device_status, kStatusWaitTimeout);
    return false;
}

}  // namespace mbc
