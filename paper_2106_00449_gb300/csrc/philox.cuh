// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11) and Box-Muller normals, shared by
// the W / W-tilde draws (geometry.cu) and the FCM stress (fcm.cu).  Counter (k/2, owner,
// step, stream), key (seed low, seed high); normal k is component k % 2 of counter k / 2.
#pragma once

#include <cuda_runtime.h>

namespace gdc {

__device__ inline uint4 philox4x32_10(uint4 ctr, uint2 key) {
    const unsigned int M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const unsigned int W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        if (rnd > 0) {
            key.x += W0;
            key.y += W1;
        }
        const unsigned int hi0 = __umulhi(M0, ctr.x), lo0 = M0 * ctr.x;
        const unsigned int hi1 = __umulhi(M1, ctr.z), lo1 = M1 * ctr.z;
        ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    }
    return ctr;
}

__device__ inline double normal_from(uint4 x, int comp) {
    const double u = (double)(x.x >> 5) * 7.450580596923828125e-9 + (double)(x.y >> 6) * 1.1102230246251565404e-16;
    const double v = (double)(x.z >> 5) * 7.450580596923828125e-9 + (double)(x.w >> 6) * 1.1102230246251565404e-16;
    const double rad = sqrt(-2.0 * log1p(-u));
    const double ang = 2.0 * 3.141592653589793 * v;
    return comp == 0 ? rad * cos(ang) : rad * sin(ang);
}

// The two normals of a Philox output in FP32: the same uniforms as normal_from, with 1 - u
// formed from the integer words so that it never rounds to zero (no log(0)).
__device__ inline void normals_f32(uint4 x, float& n0, float& n1) {
    const float om = (float)((1u << 27) - 1u - (x.x >> 5)) * 7.450580596923828125e-9f +
                     (float)((1u << 26) - (x.y >> 6)) * 1.1102230246251565404e-16f;
    const float v = (float)(x.z >> 5) * 7.450580596923828125e-9f + (float)(x.w >> 6) * 1.1102230246251565404e-16f;
    const float rad = sqrtf(-2.f * logf(om));
    float s, c;
    sincospif(2.f * v, &s, &c);
    n0 = rad * c;
    n1 = rad * s;
}

}  // namespace gdc
