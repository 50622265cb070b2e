// Pair force between blobs of different bodies, shared by the all-pairs tile kernels
// (rpy.cu) and the cell-list kernel (cells.cu).
//
// F(r) = -dU_k/dr (F > 0 pushes the blobs apart) for
//   k = 0: the soft sphere of Eq. (soft_sphere_potential), U = U0 exp((2a - r)/b) for
//          r >= 2a, whose force is A exp(-(r - 2a)/b) with A = U0/b;
//   k = 1: U_1 = U - phi_{3a}, k = 2: U_2 = U - phi_{3a} + phi_{7a/2} (Sec. 6.4), with the
//          Gaussian wells phi_c(r) = A_w exp(-((r - c)/lambda)^2), whose force is
//          -dphi_c/dr = (2 A_w/lambda) x exp(-x^2), x = (r - c)/lambda.
// Every potential continues linearly below 2a, so the force there is the force at 2a.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace gdc {

template <typename T>
struct ForceK {
    T A;       // soft-sphere force amplitude U0/b (0: no soft sphere)
    T inv_b;   // 1/b
    T two_a;   // 2a
    T rc2;     // squared cutoff
    T wA2;     // 2 A_w / lambda
    T inv_lam; // 1/lambda
    T c1, c2;  // well centres 3a and 7a/2
    int pot;   // 0, 1, 2 as above
};

__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }

template <typename T>
__device__ __forceinline__ T pair_force(T r, const ForceK<T>& k) {
    const T rr = r > k.two_a ? r : k.two_a;
    T F = k.A > T(0) ? k.A * exp_t(-(rr - k.two_a) * k.inv_b) : T(0);
    if (k.pot >= 1) {
        const T x = (rr - k.c1) * k.inv_lam;
        F -= k.wA2 * x * exp_t(-x * x);
    }
    if (k.pot == 2) {
        const T x = (rr - k.c2) * k.inv_lam;
        F += k.wA2 * x * exp_t(-x * x);
    }
    return F;
}

// Cutoff of the pair force: the soft sphere below 2.4e-16 A (36 decay lengths past 2a), the
// wells below 2e-15 (2 A_w / lambda) (six widths past the outer centre).
inline double force_cutoff(const gdc_params& p) {
    double rc = 0.0;
    if (p.rep_A > 0.0) rc = 2.0 * p.a + 36.0 * p.rep_b;
    if (p.potential > 0 && p.well_A > 0.0) rc = std::max(rc, (p.potential == 2 ? 3.5 : 3.0) * p.a + 6.0 * p.well_lambda);
    return rc;
}

inline bool forces_on(const gdc_params& p) { return p.rep_A > 0.0 || (p.potential > 0 && p.well_A > 0.0); }

template <typename T>
inline ForceK<T> force_constants(const gdc_params& p) {
    const double rc = force_cutoff(p);
    const bool wells = p.potential > 0 && p.well_A > 0.0;
    ForceK<T> k;
    k.A = (T)p.rep_A;
    k.inv_b = p.rep_A > 0.0 ? (T)(1.0 / p.rep_b) : T(0);
    k.two_a = (T)(2.0 * p.a);
    k.rc2 = (T)(rc * rc);
    k.wA2 = wells ? (T)(2.0 * p.well_A / p.well_lambda) : T(0);
    k.inv_lam = wells ? (T)(1.0 / p.well_lambda) : T(0);
    k.c1 = (T)(3.0 * p.a);
    k.c2 = (T)(3.5 * p.a);
    k.pot = wells ? p.potential : 0;
    return k;
}

}  // namespace gdc
