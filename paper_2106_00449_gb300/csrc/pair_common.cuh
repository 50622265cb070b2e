// Device helpers shared by the FP32 pair kernels: packed f32x2 arithmetic, the RPY
// constants in FP32, and bulk (TMA) tile copies into shared memory completed on an
// mbarrier with bounded waits.
#pragma once

#include "common.cuh"

namespace gdc {

struct RpyConst32 {
    float c23;     // 2a^2/3
    float c2;      // 2a^2
    float four_a2; // 4a^2
    float cA;      // 4/(3a)
    float c9;      // 9/(32a)
    float cB;      // 1/(8a^2)
};

static inline RpyConst32 rpy_const32(double a) {
    return RpyConst32{(float)(2.0 * a * a / 3.0), (float)(2.0 * a * a), (float)(4.0 * a * a),
                      (float)(4.0 / (3.0 * a)),   (float)(9.0 / (32.0 * a)), (float)(1.0 / (8.0 * a * a))};
}

// Packed FP32 pairs (Blackwell f32x2 instructions): lane .x and .y of a float2 hold
// the same quantity for two different targets.
__device__ __forceinline__ unsigned long long f2u(float2 a) { return *reinterpret_cast<unsigned long long*>(&a); }
__device__ __forceinline__ float2 u2f(unsigned long long a) { return *reinterpret_cast<float2*>(&a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
    return u2f(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_tile_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    unsigned long long state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state) : "r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
    (void)state;
}

// Bounded wait for the phase `parity` of an mbarrier: false after `polls` unsuccessful
// polls (none at all when polls <= 0).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int polls = GDC_WAIT_POLLS) {
    for (int i = 0; i < polls; ++i) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace gdc
