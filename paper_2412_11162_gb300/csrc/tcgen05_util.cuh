// Small helpers of the library's tcgen05 kernels (sm_103a): shared-memory
// addresses, the shared-memory matrix descriptor of the canonical K-major
// layout without swizzling, TF32 rounding, and the iteration limit of every
// bounded mbarrier wait.  Encodings follow the PTX ISA's tcgen05 chapter.
#pragma once

#include <cstdint>

namespace pmlbie {
namespace tcu {

// iteration limit of a bounded mbarrier wait (then the kernel records an
// error and returns)
constexpr long long kWaitLimit = 1ll << 24;

// Shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), fixed field 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

}  // namespace tcu
}  // namespace pmlbie
