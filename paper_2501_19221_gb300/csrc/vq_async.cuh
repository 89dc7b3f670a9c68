// vq_async.cuh -- mbarriers and 1-D bulk copies (global -> shared) for
// kernels that stage their operands with the copy engine (the batched
// tensor-core kernel). Every wait is bounded: it gives up after
// kAsyncWaitCycles (about two seconds) or when another thread of the launch
// already gave up, and records its code in the error word.
#pragma once

#include <cstdint>

namespace vqa {

constexpr long long kAsyncWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t c) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void mb_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t* b, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(par)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t par, int* err, int code) {
    const long long t0 = clock64();
    uint32_t spins = 0;
    while (!mb_try(b, par)) {
        if ((++spins & 1023u) == 0) {
            if (*(volatile int*)err) return false;
            if (clock64() - t0 > kAsyncWaitCycles) {
                atomicOr(err, code);
                return false;
            }
        }
    }
    return true;
}
// Makes the barrier initialisation visible to the copy engine.
__device__ __forceinline__ void mb_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// bytes (a multiple of 16) from 16-byte aligned global src to 16-byte aligned
// shared dst; completes `bytes` of the barrier's expected transactions
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// The same copy with an L2 cache policy (e.g. evict-first for data that
// streams through once).
__device__ __forceinline__ void bulk_g2s_stream(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                uint64_t pol) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 ::"r"(su32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(su32(bar)), "l"(pol)
                 : "memory");
}

}  // namespace vqa
