// Double-float (df) arithmetic on the FP32 pipes for the accurate residual products of the
// FP32-mixed mobility solve: a value is an unevaluated sum hi + lo of two floats (about 48
// significant bits).  The error-free transformations are Knuth's two-sum, Dekker's fast
// two-sum and the FMA-based exact product; the _rn intrinsics are never fused into FMAs by
// the compiler, which these transformations rely on.
#pragma once

#include "common.cuh"

namespace gdc {

struct df { float h, l; };

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df df_fast(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df x, df y) {
    df s = df_two_sum(x.h, y.h);
    return df_fast(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df{-y.h, -y.l}); }
__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = fmaf(x.h, y.h, -p);                 // exact rounding error of the product
    e = fmaf(x.h, y.l, fmaf(x.l, y.h, e));
    return df_fast(p, e);
}
__device__ __forceinline__ df df_from(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to(df x) { return (double)x.h + (double)x.l; }

// 1/sqrt(x) to double-float accuracy: one Newton step from the FP32 estimate,
// y1 = y (1 - (x y^2 - 1)/2), with the residual x y^2 - 1 formed from exact products.
__device__ __forceinline__ df df_rsqrt(df x) {
    const float y = rsqrtf(x.h);
    const float yy = __fmul_rn(y, y), yye = fmaf(y, y, -yy);
    const float h = __fadd_rn(fmaf(x.h, yy, -1.f), fmaf(x.h, yye, __fmul_rn(x.l, yy)));
    return df_fast(y, __fmul_rn(__fmul_rn(-0.5f, y), h));
}

struct RpyConstDF {
    df c23, c2, cA, c9, cB;
    df four_a2;   // 4a^2
};

inline df df_from_host(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

inline RpyConstDF df_constants(double a) {
    RpyConstDF k;
    k.c23 = df_from_host(2.0 * a * a / 3.0);
    k.c2 = df_from_host(2.0 * a * a);
    k.cA = df_from_host(4.0 / (3.0 * a));
    k.c9 = df_from_host(9.0 / (32.0 * a));
    k.cB = df_from_host(1.0 / (8.0 * a * a));
    k.four_a2 = df_from_host(4.0 * a * a);
    return k;
}

// ---- FP64 RPY pair kernel -----------------------------------------------------

}  // namespace gdc
