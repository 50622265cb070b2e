// The wall correction of the RPY tensor for blobs above a no-slip wall at z = 0 (the setting
// of the paper's RPY runs, Sec. 4.1 and Sec. 6.2), one blob pair at a time.
//
// Wall correction.  For a target blob at x and a source blob at y = (y1, y2, h), let
// R = (x1 - y1, x2 - y2, x3 + h) (x minus the mirror image of y), r = |R|.  The image system
// of a point force above a wall (Stokeslet at the mirror point with a source dipole and a
// Stokes doublet, whose strengths carry h), averaged over both spheres' surfaces with the
// Faxen operators (1 + a^2/6 Lap_x)(1 + a^2/6 Lap_y), reduces for a blob pair to
//   8 pi eta W lambda = al0 lambda + be0 R (R . lambda)
//                     + 2 [al m + be R (R . m) + ga e3 (R . m) + ep R m_3 + ze e3 m_3],
// m = (lambda_1, lambda_2, -lambda_3) (the mirror acts on the source's force), with
//   al0 = -1/r - 2a^2/(3r^3)                  be0 = -1/r^3 + 2a^2/r^5
//   al  = h^2/r^3 - h R3/r^3 + a^2 R3^2/r^5 + a^4/(3r^5) - 5a^4 R3^2/(3r^7)
//   be  = -3h^2/r^5 + 3h R3/r^5 - 5a^2 R3^2/r^7 - 5a^4/(3r^7) + 35a^4 R3^2/(3r^9)
//   ga  = h/r^3 - 10a^4 R3/(3r^7)             ep = -h/r^3 + 2a^2 R3/r^5 - 10a^4 R3/(3r^7)
//   ze  = 2a^4/(3r^5).
// The self pair (x = y, R = (0, 0, 2h)) gives the classical wall self-mobility
// 1 - 9a/(16h) + a^3/(8h^3) - a^5/(16h^5) parallel and 1 - 9a/(8h) + a^3/(2h^3) - a^5/(8h^5)
// normal to the wall (units of 1/(6 pi eta a)).  The free-space part is the unbounded RPY
// product of the other kernels, so the wall mobility is that product plus W over every pair
// of a suspension, same-body and self pairs included.  Valid for blob centres above z = a.
#pragma once

#include "common.cuh"

namespace gdc {

template <typename T>
__device__ __forceinline__ void wall_pair(T R1, T R2, T R3, T h, T a2, T l1, T l2, T l3, T& u1, T& u2, T& u3) {
    const T r2 = R1 * R1 + R2 * R2 + R3 * R3;
    const T i1 = T(1) / sqrt(r2);
    const T i2 = i1 * i1;
    const T i3 = i1 * i2, i5 = i3 * i2, i7 = i5 * i2, i9 = i7 * i2;
    const T a4 = a2 * a2, R33 = R3 * R3;
    const T al0 = -i1 - T(2.0 / 3.0) * a2 * i3;
    const T be0 = -i3 + T(2) * a2 * i5;
    const T al = h * h * i3 - h * R3 * i3 + a2 * R33 * i5 + T(1.0 / 3.0) * a4 * i5 - T(5.0 / 3.0) * a4 * R33 * i7;
    const T be = T(-3) * h * h * i5 + T(3) * h * R3 * i5 - T(5) * a2 * R33 * i7 - T(5.0 / 3.0) * a4 * i7 +
                 T(35.0 / 3.0) * a4 * R33 * i9;
    const T ga = h * i3 - T(10.0 / 3.0) * a4 * R3 * i7;
    const T ep = -h * i3 + T(2) * a2 * R3 * i5 - T(10.0 / 3.0) * a4 * R3 * i7;
    const T ze = T(2.0 / 3.0) * a4 * i5;
    const T m3 = -l3;
    const T Rl = R1 * l1 + R2 * l2 + R3 * l3;
    const T Rm = R1 * l1 + R2 * l2 + R3 * m3;
    u1 += al0 * l1 + be0 * R1 * Rl + T(2) * (al * l1 + be * R1 * Rm + ep * R1 * m3);
    u2 += al0 * l2 + be0 * R2 * Rl + T(2) * (al * l2 + be * R2 * Rm + ep * R2 * m3);
    u3 += al0 * l3 + be0 * R3 * Rl + T(2) * (al * m3 + be * R3 * Rm + ga * Rm + ep * R3 * m3 + ze * m3);
}

}  // namespace gdc
