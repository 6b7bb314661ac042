// Device helpers shared by the tcgen05 kernels: shared-memory addresses and
// matrix descriptors, and bounded mbarrier waits (every wait gives up after
// a number of polls or a time limit, so no kernel can spin forever).
#pragma once

#include <cstdint>

namespace mpg {

constexpr uint32_t TC_SPIN = 1u << 24;
constexpr uint64_t TC_WAIT_NS = 4000000000ull;   // 4 s

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the layout a SWIZZLE_128B tensor map writes).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of parity `parity`; false after TC_SPIN polls or
// TC_WAIT_NS nanoseconds, or when another role has raised the abort flag
// (abort_flag == nullptr: teardown wait for asynchronous work already in
// flight, which ignores the flag).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* abort_flag,
                                          uint64_t limit_ns = TC_WAIT_NS) {
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < TC_SPIN; i++) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255) == 255) {
            if (abort_flag && *abort_flag) return false;
            const uint64_t t = global_ns();
            if (!t0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
    return false;
}

__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) { return mbar_wait(bar, parity, nullptr); }

}  // namespace mpg
