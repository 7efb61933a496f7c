// Device helpers shared by the tcgen05 kernels: shared-memory addresses,
// bounded mbarrier waits, tcgen05 thread-sync fences and the shared-memory
// matrix descriptor of a K-major operand in the 128-byte swizzled layout.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tn {

// limit of every bounded wait of the tcgen05 kernels
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false (and the error flag set) after `limit` ns, or at once
// when another thread has already given up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err,
                                          unsigned long long limit) {
    if (mbar_try(bar, parity)) return true;
    unsigned long long t0 = gtimer();
    while (!mbar_try(bar, parity)) {
        if (*(volatile int *)err) return false;
        if (gtimer() - t0 > limit) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}
// wait for asynchronous work that completes on its own (TMA transfers and
// MMAs already issued) before the CTA releases its shared memory and TMEM;
// bounded by TC_WAIT_NS, regardless of the error flag
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity, int *err) {
    if (mbar_try(bar, parity)) return true;
    unsigned long long t0 = gtimer();
    while (!mbar_try(bar, parity)) {
        if (gtimer() - t0 > TC_WAIT_NS) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}


}  // namespace tn
