// Rigid-body state kernels: blob positions (Sec. 2), Philox draws (Sec. 3 step 1),
// the RFD/FD perturbations and divergence (Sec. 3 step 3, Eqs. FD and rfd_div), the mid-step
// and final updates (Sec. 3 steps 4 and 6), and the right-hand side of Eq. (step5).
#include "common.cuh"
#include "philox.cuh"

namespace gdc {

// ---- configuration: rotations and blob positions --------------------------

__global__ void k_body_rot(int NB, const double* __restrict__ Y, const double* __restrict__ q,
                           double* __restrict__ Rb, double* __restrict__ Yc) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NB) return;
    double R[9];
    quat_to_R(q + 4 * p, R);
#pragma unroll
    for (int k = 0; k < 9; ++k) Rb[9 * p + k] = R[k];
    Yc[3 * p] = Y[3 * p];
    Yc[3 * p + 1] = Y[3 * p + 1];
    Yc[3 * p + 2] = Y[3 * p + 2];
}

__global__ void k_blob_pos(int NBL, const int* __restrict__ blob_body, const int* __restrict__ blob_susp,
                           const int* __restrict__ body_tmpl, const long long* __restrict__ body_blob_off,
                           const int* __restrict__ tmpl_off, const double* __restrict__ tmpl_xyz,
                           const double* __restrict__ Y, const double* __restrict__ Rb,
                           const double* __restrict__ ref, double* __restrict__ r,
                           float4* __restrict__ spos, double4_32a* __restrict__ spos64) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const int p = blob_body[i];
    const int t = body_tmpl[p];
    const long long loc = i - body_blob_off[p];
    const double* b = tmpl_xyz + 3 * (tmpl_off[t] + loc);
    const double* R = Rb + 9 * p;
    double x = Y[3 * p] + R[0] * b[0] + R[1] * b[1] + R[2] * b[2];
    double y = Y[3 * p + 1] + R[3] * b[0] + R[4] * b[1] + R[5] * b[2];
    double z = Y[3 * p + 2] + R[6] * b[0] + R[7] * b[1] + R[8] * b[2];
    r[3 * i] = x;
    r[3 * i + 1] = y;
    r[3 * i + 2] = z;
    const int s = blob_susp[i];
    const double rx = x - ref[3 * s], ry = y - ref[3 * s + 1], rz = z - ref[3 * s + 2];
    const float pb = __int_as_float(p);
    spos[i] = make_float4((float)rx, (float)ry, (float)rz, pb);
    spos64[i] = make_double4_32a(rx, ry, rz, (double)p);
}

void load_config(gdc_ctx* c, const double* Y, const double* q) {
    ++c->n_launch, k_body_rot<<<ceil_div(c->NB, 128), 128, 0, c->stream>>>(c->NB, Y, q, c->Rb, c->Yc);
    ++c->n_launch, k_blob_pos<<<ceil_div(c->NBL, 128), 128, 0, c->stream>>>(
        c->NBL, c->blob_body, c->blob_susp, c->body_tmpl, c->body_blob_off, c->tmpl_off, c->tmpl_xyz,
        Y, c->Rb, c->ref, c->r, c->spos, c->spos64);
    launch_near_build(c);   // pairs closer than 2a, corrected after every FP32 product
    if (c->p.wall) launch_wall_blocks(c);   // a wall: per-body blocks depend on the configuration
}

// stream 0: 3 draws per blob; stream 1: 6 draws per body.  Counter (k/2, s, step, stream).
__global__ void k_normals(long long total, int per, const int* __restrict__ owner_susp,
                          const long long* __restrict__ susp_off, unsigned long long seed,
                          unsigned long long step, const unsigned long long* __restrict__ step_dev,
                          unsigned int stream, double* __restrict__ out) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    if (step_dev) step = *step_dev;   // graph mode: the counter lives in device memory
    const int s = owner_susp[e / per];
    const long long k = e - per * susp_off[s];
    const uint4 ctr = make_uint4((unsigned int)(k >> 1), (unsigned int)s, (unsigned int)(step & 0xffffffffull), stream);
    const uint2 key = make_uint2((unsigned int)(seed & 0xffffffffull), (unsigned int)(seed >> 32));
    out[e] = normal_from(philox4x32_10(ctr, key), (int)(k & 1));
}

void launch_normals(gdc_ctx* c, unsigned long long step, int stream, double* out, const unsigned long long* step_dev) {
    if (stream == 0) {
        long long total = 3LL * c->NBL;
        ++c->n_launch, k_normals<<<ceil_div(total, 256), 256, 0, c->stream>>>(total, 3, c->blob_susp, c->susp_blob_off,
                                                               c->p.seed, step, step_dev, 0u, out);
    } else {
        long long total = 6LL * c->NB;
        ++c->n_launch, k_normals<<<ceil_div(total, 256), 256, 0, c->stream>>>(total, 6, c->body_susp, c->susp_body_off,
                                                               c->p.seed, step, step_dev, 1u, out);
    }
}

// ---- perturbations and updates -----------------------------------------------

// RFD state of Eq. (rfd_div) with the footnote's length scale: Y + delta L_p W~_t, exp(delta W~_r) * q.
__global__ void k_perturb(int NB, const double* __restrict__ Y, const double* __restrict__ q,
                          const double* __restrict__ Wt, const double* __restrict__ L, double delta,
                          double* __restrict__ Yo, double* __restrict__ qo) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NB) return;
    const double dl = delta * L[p];
    for (int k = 0; k < 3; ++k) Yo[3 * p + k] = Y[3 * p + k] + dl * Wt[6 * p + k];
    double u[3] = {delta * Wt[6 * p + 3], delta * Wt[6 * p + 4], delta * Wt[6 * p + 5]};
    double qn[4];
    quat_exp_mul(u, q + 4 * p, qn);
    for (int k = 0; k < 4; ++k) qo[4 * p + k] = qn[k];
}

void launch_perturb(gdc_ctx* c, const double* Y, const double* q, const double* Wt, double delta,
                    double* Yo, double* qo) {
    ++c->n_launch, k_perturb<<<ceil_div(c->NB, 128), 128, 0, c->stream>>>(c->NB, Y, q, Wt, c->body_L, delta, Yo, qo);
}

// FD state of Eq. (FD): coordinate `coord` of the body with local index p_local of every suspension.
__global__ void k_perturb_one(int NB, const double* __restrict__ Y, const double* __restrict__ q,
                              const int* __restrict__ body_susp, const long long* __restrict__ susp_body_off,
                              const double* __restrict__ L, int p_local, int coord, double delta,
                              double* __restrict__ Yo, double* __restrict__ qo) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NB) return;
    const bool hit = (p - susp_body_off[body_susp[p]]) == p_local;
    for (int k = 0; k < 3; ++k) Yo[3 * p + k] = Y[3 * p + k] + ((hit && coord == k) ? delta * L[p] : 0.0);
    if (hit && coord >= 3) {
        double u[3] = {0.0, 0.0, 0.0};
        u[coord - 3] = delta;
        double qn[4];
        quat_exp_mul(u, q + 4 * p, qn);
        for (int k = 0; k < 4; ++k) qo[4 * p + k] = qn[k];
    } else {
        for (int k = 0; k < 4; ++k) qo[4 * p + k] = q[4 * p + k];
    }
}

void launch_perturb_one(gdc_ctx* c, const double* Y, const double* q, int p_local, int coord,
                        double delta, double* Yo, double* qo) {
    ++c->n_launch, k_perturb_one<<<ceil_div(c->NB, 128), 128, 0, c->stream>>>(c->NB, Y, q, c->body_susp, c->susp_body_off,
                                                               c->body_L, p_local, coord, delta, Yo, qo);
}

// x -> x + h V with q -> exp(h Omega) * q; h is multiplied by nu[s] when nu is given (Sec. 3 steps 4, 6).
// guard (graph mode): when given and zero the state is left as it is (an earlier stage failed)
__global__ void k_advance(int NB, const double* __restrict__ Y, const double* __restrict__ q,
                          const double* __restrict__ V, double h, const double* __restrict__ nu,
                          const int* __restrict__ body_susp, const int* __restrict__ guard, double* __restrict__ Yo,
                          double* __restrict__ qo) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NB) return;
    if (guard && *guard == 0) return;
    const double hp = nu ? h * nu[body_susp[p]] : h;
    double y0 = Y[3 * p] + hp * V[6 * p], y1 = Y[3 * p + 1] + hp * V[6 * p + 1], y2 = Y[3 * p + 2] + hp * V[6 * p + 2];
    double u[3] = {hp * V[6 * p + 3], hp * V[6 * p + 4], hp * V[6 * p + 5]};
    double qn[4];
    quat_exp_mul(u, q + 4 * p, qn);
    Yo[3 * p] = y0;
    Yo[3 * p + 1] = y1;
    Yo[3 * p + 2] = y2;
    for (int k = 0; k < 4; ++k) qo[4 * p + k] = qn[k];
}

void launch_advance(gdc_ctx* c, const double* Y, const double* q, const double* V, double h,
                    const double* nu, double* Yo, double* qo, const int* guard) {
    ++c->n_launch, k_advance<<<ceil_div(c->NB, 128), 128, 0, c->stream>>>(c->NB, Y, q, V, h, nu, c->body_susp, guard,
                                                                          Yo, qo);
}

// One block per suspension; fixed-order block reduction (deterministic).
__global__ void k_rfd_div(const long long* __restrict__ susp_body_off, const double* __restrict__ Wt,
                          const double* __restrict__ calV, const double* __restrict__ calVt,
                          const double* __restrict__ L, double delta, double dt, double* __restrict__ nu) {
    const int s = blockIdx.x;
    double acc = 0.0;
    for (long long p = susp_body_off[s] + threadIdx.x; p < susp_body_off[s + 1]; p += blockDim.x) {
        double t = 0.0, r = 0.0;
        for (int k = 0; k < 3; ++k) t += Wt[6 * p + k] * (calVt[6 * p + k] - calV[6 * p + k]);
        for (int k = 3; k < 6; ++k) r += Wt[6 * p + k] * (calVt[6 * p + k] - calV[6 * p + k]);
        acc += t / (delta * L[p]) + r / delta;
    }
    __shared__ double sh[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) nu[s] = 1.0 + 0.5 * dt * v;
    }
}

void launch_rfd_div(gdc_ctx* c, const double* Wt, const double* calV, const double* calVt,
                    double delta, double dt, double* nu) {
    ++c->n_launch, k_rfd_div<<<c->S, 256, 0, c->stream>>>(c->susp_body_off, Wt, calV, calVt, c->body_L, delta, dt, nu);
}

__global__ void k_fd_accum(int S, const long long* __restrict__ susp_body_off, const double* __restrict__ calV,
                           const double* __restrict__ calVp, const double* __restrict__ L, int p_local,
                           int coord, double delta, double* __restrict__ div, int first) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double prev = first ? 0.0 : div[s];
    const long long p = susp_body_off[s] + p_local;
    if (p < susp_body_off[s + 1]) {
        const double h = coord < 3 ? delta * L[p] : delta;
        prev += (calVp[6 * p + coord] - calV[6 * p + coord]) / h;
    }
    div[s] = prev;
}

void launch_fd_accum(gdc_ctx* c, const double* calV, const double* calVp, int p_local, int coord,
                     double delta, double* div, int first) {
    ++c->n_launch, k_fd_accum<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, c->susp_body_off, calV, calVp, c->body_L,
                                                           p_local, coord, delta, div, first);
}

__global__ void k_nu(int S, const double* __restrict__ div, double dt, double* __restrict__ nu) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) nu[s] = 1.0 + 0.5 * dt * div[s];
}

void launch_nu_from_div(gdc_ctx* c, const double* div, double dt, double* nu) {
    ++c->n_launch, k_nu<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, div, dt, nu);
}

// ---- right-hand side and solution layout -----------------------------------------

// b = [-vbrev - u_inf(r); -FT] in the saddle layout (Eq. step5, with the background flow reading).
__global__ void k_rhs_blob(int NBL, const int* __restrict__ blob_gm, const double* __restrict__ vb,
                           const double* __restrict__ r, double shear, double* __restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const long long o = blob_gm[i];
    double v0 = vb ? vb[3 * i] : 0.0, v1 = vb ? vb[3 * i + 1] : 0.0, v2 = vb ? vb[3 * i + 2] : 0.0;
    v0 += shear * r[3 * i + 1];
    b[o] = -v0;
    b[o + 1] = -v1;
    b[o + 2] = -v2;
}

__global__ void k_rhs_body(int NB, const int* __restrict__ body_gm, const double* __restrict__ FT,
                           double* __restrict__ b) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NB) return;
    const long long o = body_gm[p];
    for (int k = 0; k < 6; ++k) b[o + k] = FT ? -FT[6 * p + k] : 0.0;
}

void launch_rhs(gdc_ctx* c, const double* vbrev, const double* FT, double* b) {
    ++c->n_launch, k_rhs_blob<<<ceil_div(c->NBL, 128), 128, 0, c->stream>>>(c->NBL, c->blob_gm, vbrev, c->r, c->p.shear_rate, b);
    ++c->n_launch, k_rhs_body<<<ceil_div(c->NB, 128), 128, 0, c->stream>>>(c->NB, c->body_gm, FT, b);
}

__global__ void k_scatter_V(int NB, const int* __restrict__ body_gm, const double* __restrict__ x,
                            double* __restrict__ V) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NB) return;
    for (int k = 0; k < 6; ++k) V[6 * p + k] = x[body_gm[p] + k];
}

__global__ void k_scatter_lam(int NBL, const int* __restrict__ blob_gm, const double* __restrict__ x,
                              double* __restrict__ lam) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    for (int k = 0; k < 3; ++k) lam[3 * i + k] = x[blob_gm[i] + k];
}

void launch_scatter_solution(gdc_ctx* c, const double* x, double* V, double* lambda) {
    if (V) ++c->n_launch, k_scatter_V<<<ceil_div(c->NB, 128), 128, 0, c->stream>>>(c->NB, c->body_gm, x, V);
    if (lambda) ++c->n_launch, k_scatter_lam<<<ceil_div(c->NBL, 128), 128, 0, c->stream>>>(c->NBL, c->blob_gm, x, lambda);
}

}  // namespace gdc

namespace gdc {

// Reference point of each suspension (mean body centre): the pair kernels take
// positions relative to it, which keeps FP32 coordinates small.
__global__ void k_ref(const long long* __restrict__ susp_body_off, const double* __restrict__ Y, double* __restrict__ ref) {
    const int s = blockIdx.x;
    __shared__ double sh[3][32];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const long long lo = susp_body_off[s], hi = susp_body_off[s + 1];
    for (long long p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        a0 += Y[3 * p];
        a1 += Y[3 * p + 1];
        a2 += Y[3 * p + 2];
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a0;
        sh[1][threadIdx.x >> 5] = a1;
        sh[2][threadIdx.x >> 5] = a2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double acc = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += sh[threadIdx.x][w];
        ref[3 * s + threadIdx.x] = hi > lo ? acc / (double)(hi - lo) : 0.0;
    }
}

void launch_ref(gdc_ctx* c, const double* Y) {
    ++c->n_launch, k_ref<<<c->S, 256, 0, c->stream>>>(c->susp_body_off, Y, c->ref);
}

}  // namespace gdc
