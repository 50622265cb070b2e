// Blobs above a no-slip wall at z = 0 (Sec. 4.1, Sec. 6.2): the wall correction of the RPY
// product over every pair of a suspension (the pair term is in wall_pair.cuh; the per-body
// blocks of the preconditioners are set up in body.cu), and the wall and gravity forces of
// Sec. 6.2.
#include <algorithm>

#include "common.cuh"
#include "wall_pair.cuh"

namespace gdc {

constexpr int WALL_TILE = 128;   // targets per block and sources per shared-memory tile

// y_i += W lambda (all blobs j of i's suspension), one thread per target, sources staged in
// shared memory; items are (suspension, first target).  Positions are absolute FP64 (the
// wall term needs heights); differences are taken in FP64 and the pair term is evaluated in
// T.  x and y hold 3 doubles per blob, or the saddle layout through blob_gm (gm = 1).
template <typename T>
__global__ void __launch_bounds__(WALL_TILE) k_wall_apply(const int2* __restrict__ items,
                                                          const long long* __restrict__ susp_blob_off,
                                                          const double* __restrict__ r, const double* __restrict__ x,
                                                          double* __restrict__ y, int gm, const int* __restrict__ blob_gm,
                                                          double a, double c0, const int* __restrict__ active) {
    __shared__ double sp[WALL_TILE][3];
    __shared__ T sl[WALL_TILE][3];
    const int2 it = items[blockIdx.x];
    if (active && !active[it.x]) return;   // a suspension whose Krylov loop has stopped
    const long long b0 = susp_blob_off[it.x], ns = susp_blob_off[it.x + 1] - b0;
    const long long i = b0 + it.y + threadIdx.x;
    const bool own = it.y + threadIdx.x < ns;
    double xi = 0.0, yi = 0.0, zi = 0.0;
    if (own) {
        xi = r[3 * i];
        yi = r[3 * i + 1];
        zi = r[3 * i + 2];
    }
    const T a2 = T(a * a);
    T u1 = T(0), u2 = T(0), u3 = T(0);
    for (long long j0 = 0; j0 < ns; j0 += WALL_TILE) {
        __syncthreads();
        const long long j = j0 + threadIdx.x;
        if (j < ns) {
            const long long g = b0 + j;
            const long long o = gm ? (long long)blob_gm[g] : 3 * g;
            sp[threadIdx.x][0] = r[3 * g];
            sp[threadIdx.x][1] = r[3 * g + 1];
            sp[threadIdx.x][2] = r[3 * g + 2];
            sl[threadIdx.x][0] = (T)x[o];
            sl[threadIdx.x][1] = (T)x[o + 1];
            sl[threadIdx.x][2] = (T)x[o + 2];
        }
        __syncthreads();
        const int n = (int)std::min<long long>(WALL_TILE, ns - j0);
        if (own)
            for (int k = 0; k < n; ++k)
                wall_pair<T>((T)(xi - sp[k][0]), (T)(yi - sp[k][1]), (T)(zi + sp[k][2]), (T)sp[k][2], a2, sl[k][0],
                             sl[k][1], sl[k][2], u1, u2, u3);
    }
    if (!own) return;
    const long long o = gm ? (long long)blob_gm[i] : 3 * i;
    y[o] += c0 * (double)u1;
    y[o + 1] += c0 * (double)u2;
    y[o + 2] += c0 * (double)u3;
}

void build_wall_items(gdc_ctx* c) {
    c->h_wall_items.clear();
    for (int s = 0; s < c->S; ++s) {
        const long long ns = c->h_blob_off[s + 1] - c->h_blob_off[s];
        for (long long t0 = 0; t0 < ns; t0 += WALL_TILE) c->h_wall_items.push_back(make_int2(s, (int)t0));
    }
}

void launch_wall_apply(gdc_ctx* c, int prec, const double* x, double* y, int gm) {
    const double c0 = 1.0 / (8.0 * 3.141592653589793 * c->p.eta);
    const int n = (int)c->h_wall_items.size();
    if (prec == GDC_FP32_MIXED)
        ++c->n_launch, k_wall_apply<float><<<n, WALL_TILE, 0, c->stream>>>(
            c->wall_items, c->susp_blob_off, c->r, x, y, gm, c->blob_gm, c->p.a, c0, c->mv_active);
    else
        ++c->n_launch, k_wall_apply<double><<<n, WALL_TILE, 0, c->stream>>>(
            c->wall_items, c->susp_blob_off, c->r, x, y, gm, c->blob_gm, c->p.a, c0, c->mv_active);
}

// ---- wall and gravity forces (Sec. 6.2) -----------------------------------------------

// f_i,z += V0 a exp(-(h - a)/b) (1/(b (h - a)) + 1/(h - a)^2) - mg / n_p: minus the derivative
// of V(h) = V0 a exp(-(h - a)/b) / (h - a) at the blob's height h, and the body's weight mg
// shared equally by its n_p blobs.  (Blobs at h <= a are flagged by the block set-up.)
__global__ void k_wall_forces(int NBL, const double* __restrict__ r, const int* __restrict__ blob_body,
                              const long long* __restrict__ body_blob_off, double V0, double b, double a,
                              double weight, double* __restrict__ f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const int p = blob_body[i];
    double fz = -weight / (double)(body_blob_off[p + 1] - body_blob_off[p]);
    const double s = r[3 * i + 2] - a;
    if (V0 != 0.0 && s > 0.0) fz += V0 * a * exp(-s / b) * (1.0 / (b * s) + 1.0 / (s * s));
    f[3 * i + 2] += fz;
}

void launch_wall_forces(gdc_ctx* c, double* fblob) {
    ++c->n_launch, k_wall_forces<<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(
        c->NBL, c->r, c->blob_body, c->body_blob_off, c->p.wall_V0, c->p.wall_b, c->p.a, c->p.body_weight, fblob);
}

}  // namespace gdc
