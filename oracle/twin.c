/*
 * Matrix-free FP64 products of the CPU twin of the gDC step (oracle/twin.py).
 * TEST INFRASTRUCTURE ONLY: the timed CPU baseline and a cross-check of the oracle at sizes
 * where the dense matrix M cannot be stored.  Plain C, one OpenMP loop over target blobs,
 * every pair evaluated directly from its formula; it shares nothing with the CUDA library.
 *
 * twin_rpy_product: u_i = sum_j M_ij lambda_j with the unbounded RPY tensor of equal blobs
 * of radius a (Sec. 4.1), overlapping form included, for d = r_i - r_j, r = |d|:
 *   r >= 2a : M_ij = 1/(8 pi eta r) [(1 + 2a^2/(3r^2)) I + (1 - 2a^2/r^2) d d^T / r^2]
 *   0<r<2a  : M_ij = 1/(6 pi eta a) [(1 - 9r/(32a)) I + (3/(32 a r)) d d^T]
 *   r == 0  : M_ij = I / (6 pi eta a)   (the self term, also for coincident blobs)
 *
 * twin_soft_forces: f_i = sum over blobs j of other bodies of F(r) d / r, with the soft
 * sphere force F(r) = A exp(-(r - 2a)/b) at max(r, 2a) (Sec. 6.3, constant below 2a);
 * pairs with (r - 2a)/b > 36 are skipped (their force is below 2.4e-16 A).
 */
#include <math.h>

void twin_rpy_product(long n, const double* r, const double* lam, double a, double eta, double* u) {
    const double pi = 3.14159265358979323846;
    const double c_far = 1.0 / (8.0 * pi * eta);
    const double c_self = 1.0 / (6.0 * pi * eta * a);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        double ux = 0.0, uy = 0.0, uz = 0.0;
        for (long j = 0; j < n; ++j) {
            const double dx = r[3 * i] - r[3 * j], dy = r[3 * i + 1] - r[3 * j + 1], dz = r[3 * i + 2] - r[3 * j + 2];
            const double lx = lam[3 * j], ly = lam[3 * j + 1], lz = lam[3 * j + 2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            double f, g;   /* u_i += f lambda_j + g (d . lambda_j) d */
            if (r2 == 0.0) {
                f = c_self;
                g = 0.0;
            } else {
                const double rr = sqrt(r2);
                if (rr >= 2.0 * a) {
                    f = c_far / rr * (1.0 + 2.0 * a * a / (3.0 * r2));
                    g = c_far / rr * (1.0 - 2.0 * a * a / r2) / r2;
                } else {
                    f = c_self * (1.0 - 9.0 * rr / (32.0 * a));
                    g = c_self * 3.0 / (32.0 * a * rr);
                }
            }
            const double dl = dx * lx + dy * ly + dz * lz;
            ux += f * lx + g * dl * dx;
            uy += f * ly + g * dl * dy;
            uz += f * lz + g * dl * dz;
        }
        u[3 * i] = ux;
        u[3 * i + 1] = uy;
        u[3 * i + 2] = uz;
    }
}

void twin_soft_forces(long n, const double* r, const int* blob_body, double A, double b, double a, double* f) {
    const double rc = 2.0 * a + 36.0 * b;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (long j = 0; j < n; ++j) {
            if (blob_body[j] == blob_body[i]) continue;
            const double dx = r[3 * i] - r[3 * j], dy = r[3 * i + 1] - r[3 * j + 1], dz = r[3 * i + 2] - r[3 * j + 2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0 || r2 > rc * rc) continue;
            const double rr = sqrt(r2);
            const double F = A * exp(-(fmax(rr, 2.0 * a) - 2.0 * a) / b);
            fx += F * dx / rr;
            fy += F * dy / rr;
            fz += F * dz / rr;
        }
        f[3 * i] = fx;
        f[3 * i + 1] = fy;
        f[3 * i + 2] = fz;
    }
}

int twin_threads(void) {
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            t = omp_get_num_threads();
#endif
        }
    }
    return t;
}
