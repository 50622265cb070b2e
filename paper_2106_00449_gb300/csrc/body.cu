// Per-body kernels: the K^T map (Eq. force_torque_balance_compact), step-2 least squares (Eq. sol_unconst with the
// closed-form K^T K of Sec. 5), the block-diagonal preconditioner P of Sec. 2.2, and
// the per-template FP64 setup of P (Cholesky of the template's RPY block).
//
// Rigidity makes every intra-body quantity a rotation of a body-frame template
// quantity: with R-hat = diag(R, ..., R) on blobs and R-tilde = diag(R, R) on
// [force; torque], K_p = R-hat K_t R-tilde^T and M_pp = R-hat M_t R-hat^T (RPY is
// rotation covariant and intra-body distances are fixed).  So M_t^-1, G_t = M_t^-1 K_t,
// N_t = (K_t^T M_t^-1 K_t)^+ and (K_t^T K_t)^+ are computed once per template in the
// body frame and applied to rotated vectors.  "^+" is the pseudo-inverse: a collinear
// body (rod) has no axial spin (its K has that null vector), which is then set to 0.
#include <algorithm>

#include "common.cuh"
#include "wall_pair.cuh"

namespace gdc {

// ---- K^T: [sum lambda_i; sum (r_i - Y_p) x lambda_i] per body, one warp per body ----

__global__ void k_body_KT(int NB, const long long* __restrict__ body_blob_off, const int* __restrict__ blob_gm,
                          const int* __restrict__ body_gm, const double* __restrict__ x, int x_gm,
                          double* __restrict__ y, int y_gm, double scale, const double* __restrict__ r,
                          const double* __restrict__ Yc) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= NB) return;
    const int p = warp;
    const double Y0 = Yc[3 * p], Y1 = Yc[3 * p + 1], Y2 = Yc[3 * p + 2];
    double f0 = 0, f1 = 0, f2 = 0, t0 = 0, t1 = 0, t2 = 0;
    for (long long i = body_blob_off[p] + lane; i < body_blob_off[p + 1]; i += 32) {
        const long long o = x_gm ? (long long)blob_gm[i] : 3 * i;
        const double l0 = x[o], l1 = x[o + 1], l2 = x[o + 2];
        const double d0 = r[3 * i] - Y0, d1 = r[3 * i + 1] - Y1, d2 = r[3 * i + 2] - Y2;
        f0 += l0;
        f1 += l1;
        f2 += l2;
        t0 += d1 * l2 - d2 * l1;
        t1 += d2 * l0 - d0 * l2;
        t2 += d0 * l1 - d1 * l0;
    }
    f0 = warp_sum(f0);
    f1 = warp_sum(f1);
    f2 = warp_sum(f2);
    t0 = warp_sum(t0);
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    if (lane == 0) {
        const long long o = y_gm ? (long long)body_gm[p] : 6LL * p;
        y[o] = scale * f0;
        y[o + 1] = scale * f1;
        y[o + 2] = scale * f2;
        y[o + 3] = scale * t0;
        y[o + 4] = scale * t1;
        y[o + 5] = scale * t2;
    }
}

void launch_body_KT(gdc_ctx* c, const double* x, int x_gm, double* y, int y_gm, double scale) {
    ++c->n_launch, k_body_KT<<<ceil_div(32LL * c->NB, 256), 256, 0, c->stream>>>(c->NB, c->body_blob_off, c->blob_gm, c->body_gm, x,
                                                                  x_gm, y, y_gm, scale, c->r, c->Yc);
}

// ---- step 2: calV_p = (K^T K)_p^+ K_p^T vbrev ----------------------------------------

__device__ inline void rotT(const double* R, const double* v, double* o) {  // o = R^T v
    o[0] = R[0] * v[0] + R[3] * v[1] + R[6] * v[2];
    o[1] = R[1] * v[0] + R[4] * v[1] + R[7] * v[2];
    o[2] = R[2] * v[0] + R[5] * v[1] + R[8] * v[2];
}

__device__ inline void rot(const double* R, const double* v, double* o) {  // o = R v
    o[0] = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
    o[1] = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
    o[2] = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
}

__global__ void k_lsq(int NB, const long long* __restrict__ body_blob_off, const int* __restrict__ body_tmpl,
                      const double* __restrict__ KtKp, const double* __restrict__ vb, const double* __restrict__ r,
                      const double* __restrict__ Yc, const double* __restrict__ Rb, double* __restrict__ calV) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= NB) return;
    const int p = warp;
    const double Y0 = Yc[3 * p], Y1 = Yc[3 * p + 1], Y2 = Yc[3 * p + 2];
    double g[6] = {0, 0, 0, 0, 0, 0};
    for (long long i = body_blob_off[p] + lane; i < body_blob_off[p + 1]; i += 32) {
        const double l0 = vb[3 * i], l1 = vb[3 * i + 1], l2 = vb[3 * i + 2];
        const double d0 = r[3 * i] - Y0, d1 = r[3 * i + 1] - Y1, d2 = r[3 * i + 2] - Y2;
        g[0] += l0;
        g[1] += l1;
        g[2] += l2;
        g[3] += d1 * l2 - d2 * l1;
        g[4] += d2 * l0 - d0 * l2;
        g[5] += d0 * l1 - d1 * l0;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) g[k] = warp_sum(g[k]);
    if (lane == 0) {
        const double* R = Rb + 9 * p;
        double gb[6], vbody[6], out[6];
        rotT(R, g, gb);
        rotT(R, g + 3, gb + 3);
        const double* A = KtKp + 36 * body_tmpl[p];
        for (int a = 0; a < 6; ++a) {
            double acc = 0.0;
            for (int b = 0; b < 6; ++b) acc += A[6 * a + b] * gb[b];
            vbody[a] = acc;
        }
        rot(R, vbody, out);
        rot(R, vbody + 3, out + 3);
        for (int k = 0; k < 6; ++k) calV[6 * p + k] = out[k];
    }
}

void launch_lsq(gdc_ctx* c, const double* vbrev, double* calV) {
    ++c->n_launch, k_lsq<<<ceil_div(32LL * c->NB, 256), 256, 0, c->stream>>>(c->NB, c->body_blob_off, c->body_tmpl, c->tmpl_KtKp,
                                                              vbrev, c->r, c->Yc, c->Rb, calV);
}

// ---- block-diagonal preconditioner, one block per body ---------------------------------
//
// Solves [M_pp -K_p; -K_p^T 0][lam; V] = [r_lam; r_V] exactly:
//   a = M^-1 r_lam,  V = -N (r_V + K^T a),  lam = a + G V   (N = (K^T M^-1 K)^+, G = M^-1 K)
// in the body frame of the template.

// LAB = false: the template's FP64 blocks in the body frame, applied to rotated vectors.
// LAB = true (blobs above a wall): each body's own blocks in the lab frame (set up by
// k_wall_blocks at every configuration), blob offsets d_i = r_i - Y_p, no rotation.
// F32: the body's M^-1 product in FP32 (the template block rounded to FP32, four interleaved
// FP32 partial sums per row added in FP64; the rest of the block solve stays FP64), for the
// inner cycles of the FP32-mixed mobility solve, whose operator already carries FP32 rounding:
// the preconditioner only has to be a fixed approximation, and the FP64 product there was
// FP64-pipe bound (1/64 of the FP32 rate).
template <bool LAB, bool F32 = false>
__global__ void __launch_bounds__(128) k_precond(const long long* __restrict__ body_blob_off, const int* __restrict__ body_tmpl,
                                                 const int* __restrict__ tmpl_n, const int* __restrict__ tmpl_off,
                                                 const long long* __restrict__ minv_off, const double* __restrict__ Minv,
                                                 const float* __restrict__ Minv32,
                                                 const double* __restrict__ Gt, const double* __restrict__ Nt,
                                                 const double* __restrict__ tmpl_xyz, const int* __restrict__ blob_gm,
                                                 const int* __restrict__ body_gm, const double* __restrict__ Rb,
                                                 const double* __restrict__ rin, double* __restrict__ zout,
                                                 const long long* __restrict__ blk_off, const double* __restrict__ r,
                                                 const double* __restrict__ Yc) {
    extern __shared__ double sh[];
    const int p = blockIdx.x;
    const int t = LAB ? p : body_tmpl[p];
    const int n = LAB ? (int)(body_blob_off[p + 1] - body_blob_off[p]) : tmpl_n[t];
    const int n3 = 3 * n;
    double* rho = sh;          // n3
    double* av = sh + n3;      // n3
    double* misc = sh + 2 * n3;  // 32
    double* bl = misc + 32;      // LAB: blob offsets d (n3)
    float* rho32 = reinterpret_cast<float*>(misc + 32);   // F32 (never with LAB): rho in FP32 (n3)
    const double ident[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    const double* R = LAB ? ident : Rb + 9 * p;
    const long long i0 = body_blob_off[p];
    if (LAB)
        for (int e = threadIdx.x; e < n3; e += blockDim.x) bl[e] = r[3 * i0 + e] - Yc[3 * p + e % 3];
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        const long long o = blob_gm[i0 + b];
        double v[3] = {rin[o], rin[o + 1], rin[o + 2]}, w[3];
        rotT(R, v, w);
        rho[3 * b] = w[0];
        rho[3 * b + 1] = w[1];
        rho[3 * b + 2] = w[2];
        if (F32) {
            rho32[3 * b] = (float)w[0];
            rho32[3 * b + 1] = (float)w[1];
            rho32[3 * b + 2] = (float)w[2];
        }
    }
    if (threadIdx.x == 0) {
        const long long o = body_gm[p];
        double v[3] = {rin[o], rin[o + 1], rin[o + 2]}, w[3];
        rotT(R, v, w);
        misc[0] = w[0];
        misc[1] = w[1];
        misc[2] = w[2];
        double v2[3] = {rin[o + 3], rin[o + 4], rin[o + 5]};
        rotT(R, v2, w);
        misc[3] = w[0];
        misc[4] = w[1];
        misc[5] = w[2];
    }
    __syncthreads();
    if (F32) {
        const float* Mi = Minv32 + minv_off[t];
        for (int row = threadIdx.x; row < n3; row += blockDim.x) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            int k = 0;
            for (; k + 3 < n3; k += 4) {   // symmetric: column-major reads are coalesced over rows
                a0 = fmaf(Mi[(long long)k * n3 + row], rho32[k], a0);
                a1 = fmaf(Mi[(long long)(k + 1) * n3 + row], rho32[k + 1], a1);
                a2 = fmaf(Mi[(long long)(k + 2) * n3 + row], rho32[k + 2], a2);
                a3 = fmaf(Mi[(long long)(k + 3) * n3 + row], rho32[k + 3], a3);
            }
            for (; k < n3; ++k) a0 = fmaf(Mi[(long long)k * n3 + row], rho32[k], a0);
            av[row] = ((double)a0 + (double)a1) + ((double)a2 + (double)a3);
        }
    } else {
        const double* Mi = Minv + (LAB ? blk_off[p] : minv_off[t]);
        for (int row = threadIdx.x; row < n3; row += blockDim.x) {
            double acc = 0.0;
            for (int k = 0; k < n3; ++k) acc = fma(Mi[(long long)k * n3 + row], rho[k], acc);  // symmetric
            av[row] = acc;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const double* b = LAB ? bl : tmpl_xyz + 3LL * tmpl_off[t];
        double g[6] = {0, 0, 0, 0, 0, 0};
        for (int i = threadIdx.x; i < n; i += 32) {
            const double a0 = av[3 * i], a1 = av[3 * i + 1], a2 = av[3 * i + 2];
            const double d0 = b[3 * i], d1 = b[3 * i + 1], d2 = b[3 * i + 2];
            g[0] += a0;
            g[1] += a1;
            g[2] += a2;
            g[3] += d1 * a2 - d2 * a1;
            g[4] += d2 * a0 - d0 * a2;
            g[5] += d0 * a1 - d1 * a0;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) g[k] = warp_sum(g[k]);
        if (threadIdx.x == 0) {
            const double* N = Nt + 36 * t;
            for (int a = 0; a < 6; ++a) {
                double acc = 0.0;
                for (int k = 0; k < 6; ++k) acc += N[6 * a + k] * (misc[k] + g[k]);
                misc[8 + a] = -acc;
            }
        }
    }
    __syncthreads();
    // G is 3n x 6, blocks back to back (templates, or LAB bodies in blob order)
    const double* Gtt = Gt + 18LL * (LAB ? body_blob_off[p] : (long long)tmpl_off[t]);
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        double lb[3];
        for (int a = 0; a < 3; ++a) {
            const int row = 3 * b + a;
            double acc = av[row];
            for (int k = 0; k < 6; ++k) acc = fma(Gtt[6LL * row + k], misc[8 + k], acc);
            lb[a] = acc;
        }
        double w[3];
        rot(R, lb, w);
        const long long o = blob_gm[i0 + b];
        zout[o] = w[0];
        zout[o + 1] = w[1];
        zout[o + 2] = w[2];
    }
    if (threadIdx.x == 0) {
        double w[3];
        const long long o = body_gm[p];
        rot(R, misc + 8, w);
        zout[o] = w[0];
        zout[o + 1] = w[1];
        zout[o + 2] = w[2];
        rot(R, misc + 11, w);
        zout[o + 3] = w[0];
        zout[o + 4] = w[1];
        zout[o + 5] = w[2];
    }
}

// ---- intra-body block of the RPY product in FP64 ---------------------------------------
//
// y_p += M_pp lambda_p with M_pp = R M_t R^T (M_t: the template's RPY block, FP64, built at
// init).  The FP32 pair kernel leaves out same-body pairs, so the large near-field terms of
// each body are added here exactly.  One block per body; x and y use the saddle layout
// (gm = 1) or 3 doubles per blob (gm = 0).
__global__ void __launch_bounds__(128) k_intra_body(const long long* __restrict__ body_blob_off, const int* __restrict__ body_tmpl,
                                                    const int* __restrict__ tmpl_n, const long long* __restrict__ minv_off,
                                                    const double* __restrict__ Mt, const int* __restrict__ blob_gm,
                                                    const double* __restrict__ Rb, const double* __restrict__ x,
                                                    double* __restrict__ y, int gm) {
    extern __shared__ double sh[];
    const int p = blockIdx.x;
    const int t = body_tmpl[p];
    const int n3 = 3 * tmpl_n[t];
    double* rho = sh;
    const double* R = Rb + 9 * p;
    const long long i0 = body_blob_off[p];
    for (int b = threadIdx.x; b < n3 / 3; b += blockDim.x) {
        const long long o = gm ? (long long)blob_gm[i0 + b] : 3 * (i0 + b);
        double v[3] = {x[o], x[o + 1], x[o + 2]}, w[3];
        rotT(R, v, w);
        rho[3 * b] = w[0];
        rho[3 * b + 1] = w[1];
        rho[3 * b + 2] = w[2];
    }
    __syncthreads();
    const double* M = Mt + minv_off[t];
    double* av = sh + n3;
    for (int row = threadIdx.x; row < n3; row += blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < n3; ++q) acc = fma(M[(long long)q * n3 + row], rho[q], acc);  // symmetric
        av[row] = acc;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n3 / 3; b += blockDim.x) {
        double w[3];
        rot(R, av + 3 * b, w);
        const long long o = gm ? (long long)blob_gm[i0 + b] : 3 * (i0 + b);
        y[o] += w[0];
        y[o + 1] += w[1];
        y[o + 2] += w[2];
    }
}

// The same block for the FP32 products, whose other terms carry FP32 rounding: M_t in FP32
// (tmpl_M32), rho rounded to FP32, each row sum split into four interleaved FP32 partial
// sums that are added in FP64; the rotations stay in FP64.  Shared memory: av (n3 doubles),
// then rho (n3 floats).
__global__ void __launch_bounds__(128) k_intra_body32(const long long* __restrict__ body_blob_off,
                                                      const int* __restrict__ body_tmpl, const int* __restrict__ tmpl_n,
                                                      const long long* __restrict__ minv_off, const float* __restrict__ Mt,
                                                      const int* __restrict__ blob_gm, const double* __restrict__ Rb,
                                                      const double* __restrict__ x, double* __restrict__ y, int gm) {
    extern __shared__ double sh[];
    const int p = blockIdx.x;
    const int t = body_tmpl[p];
    const int n3 = 3 * tmpl_n[t];
    double* av = sh;
    float* rho = reinterpret_cast<float*>(sh + n3);
    const double* R = Rb + 9 * p;
    const long long i0 = body_blob_off[p];
    for (int b = threadIdx.x; b < n3 / 3; b += blockDim.x) {
        const long long o = gm ? (long long)blob_gm[i0 + b] : 3 * (i0 + b);
        double v[3] = {x[o], x[o + 1], x[o + 2]}, w[3];
        rotT(R, v, w);
        rho[3 * b] = (float)w[0];
        rho[3 * b + 1] = (float)w[1];
        rho[3 * b + 2] = (float)w[2];
    }
    __syncthreads();
    const float* M = Mt + minv_off[t];
    for (int row = threadIdx.x; row < n3; row += blockDim.x) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int q = 0;
        for (; q + 4 <= n3; q += 4) {   // M_t is symmetric: column reads, coalesced over rows
            a0 = fmaf(M[(long long)q * n3 + row], rho[q], a0);
            a1 = fmaf(M[(long long)(q + 1) * n3 + row], rho[q + 1], a1);
            a2 = fmaf(M[(long long)(q + 2) * n3 + row], rho[q + 2], a2);
            a3 = fmaf(M[(long long)(q + 3) * n3 + row], rho[q + 3], a3);
        }
        for (; q < n3; ++q) a0 = fmaf(M[(long long)q * n3 + row], rho[q], a0);
        av[row] = ((double)a0 + (double)a1) + ((double)a2 + (double)a3);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n3 / 3; b += blockDim.x) {
        double w[3];
        rot(R, av + 3 * b, w);
        const long long o = gm ? (long long)blob_gm[i0 + b] : 3 * (i0 + b);
        y[o] += w[0];
        y[o + 1] += w[1];
        y[o + 2] += w[2];
    }
}

__global__ void k_round_f32(long long n, const double* __restrict__ a, float* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

void launch_intra_body32(gdc_ctx* c, const double* x, double* y, int gm) {
    const size_t smem = (size_t)(3 * c->max_body_blobs) * (sizeof(double) + sizeof(float));
    ++c->n_launch, k_intra_body32<<<c->NB, 128, smem, c->stream>>>(c->body_blob_off, c->body_tmpl, c->tmpl_n, c->minv_off,
                                                                   c->tmpl_M32, c->blob_gm, c->Rb, x, y, gm);
}

void launch_intra_body(gdc_ctx* c, const double* x, double* y, int gm) {
    const size_t smem = (size_t)(2 * 3 * c->max_body_blobs) * sizeof(double);
    ++c->n_launch, k_intra_body<<<c->NB, 128, smem, c->stream>>>(c->body_blob_off, c->body_tmpl, c->tmpl_n, c->minv_off,
                                                                 c->tmpl_M, c->blob_gm, c->Rb, x, y, gm);
}

// The block preconditioner for several bodies of one template per block (the items of
// k_body_tri_tb): the template's M^-1 product grouped, each element read once for all of the
// block's bodies (FP32 when F32, one accumulator per body and row), then per body (a warp
// each) the sums K^T (M^-1 rho), the 6 x 6 solve with N and the correction G V, as k_precond.
template <bool F32>
__global__ void __launch_bounds__(128) k_precond_tb(const int4* __restrict__ items, const int* __restrict__ bodies,
                                                    const long long* __restrict__ body_blob_off,
                                                    const int* __restrict__ tmpl_n, const int* __restrict__ tmpl_off,
                                                    const long long* __restrict__ minv_off,
                                                    const double* __restrict__ Minv, const float* __restrict__ Minv32,
                                                    const double* __restrict__ Gt, const double* __restrict__ Nt,
                                                    const double* __restrict__ tmpl_xyz, const int* __restrict__ blob_gm,
                                                    const int* __restrict__ body_gm, const double* __restrict__ Rb,
                                                    const double* __restrict__ rin, double* __restrict__ zout) {
    extern __shared__ double sh[];
    const int4 it = items[blockIdx.x];
    const int t = it.x, cnt = it.z;
    const int n = tmpl_n[t], n3 = 3 * n;
    double* rho = sh;                                         // [cnt][n3]
    double* av = rho + (long long)cnt * n3;                   // [cnt][n3]
    double* misc = av + (long long)cnt * n3;                  // [cnt][16]: 0-5 body rows, 8-13 V
    float* rho32 = reinterpret_cast<float*>(misc + 16 * cnt);   // [cnt][n3] (F32)
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
        const int u = e / n, b = e - u * n;
        const int p = bodies[it.y + u];
        const long long o = blob_gm[body_blob_off[p] + b];
        double v[3] = {rin[o], rin[o + 1], rin[o + 2]}, w[3];
        rotT(Rb + 9 * p, v, w);
        for (int a = 0; a < 3; ++a) {
            rho[u * n3 + 3 * b + a] = w[a];
            if (F32) rho32[u * n3 + 3 * b + a] = (float)w[a];
        }
    }
    for (int e = threadIdx.x; e < 2 * cnt; e += blockDim.x) {
        const int u = e >> 1, h = e & 1;
        const int p = bodies[it.y + u];
        const long long o = body_gm[p] + 3 * h;
        double v[3] = {rin[o], rin[o + 1], rin[o + 2]}, w[3];
        rotT(Rb + 9 * p, v, w);
        misc[16 * u + 3 * h] = w[0];
        misc[16 * u + 3 * h + 1] = w[1];
        misc[16 * u + 3 * h + 2] = w[2];
    }
    __syncthreads();
    const long long mo = minv_off[t];
    for (int row = threadIdx.x; row < n3; row += blockDim.x) {   // symmetric: coalesced over rows
        if (F32) {
            float a[GDC_TB_MAX];
#pragma unroll
            for (int u = 0; u < GDC_TB_MAX; ++u) a[u] = 0.f;
            for (int k = 0; k < n3; ++k) {
                const float f = Minv32[mo + (long long)k * n3 + row];
#pragma unroll
                for (int u = 0; u < GDC_TB_MAX; ++u)
                    if (u < cnt) a[u] = fmaf(f, rho32[u * n3 + k], a[u]);
            }
#pragma unroll
            for (int u = 0; u < GDC_TB_MAX; ++u)
                if (u < cnt) av[u * n3 + row] = (double)a[u];
        } else {
            double a[GDC_TB_MAX];
#pragma unroll
            for (int u = 0; u < GDC_TB_MAX; ++u) a[u] = 0.0;
            for (int k = 0; k < n3; ++k) {
                const double f = Minv[mo + (long long)k * n3 + row];
#pragma unroll
                for (int u = 0; u < GDC_TB_MAX; ++u)
                    if (u < cnt) a[u] = fma(f, rho[u * n3 + k], a[u]);
            }
#pragma unroll
            for (int u = 0; u < GDC_TB_MAX; ++u)
                if (u < cnt) av[u * n3 + row] = a[u];
        }
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* bx = tmpl_xyz + 3LL * tmpl_off[t];
    for (int u = warp; u < cnt; u += blockDim.x >> 5) {
        double g[6] = {0, 0, 0, 0, 0, 0};
        for (int i = lane; i < n; i += 32) {
            const double a0 = av[u * n3 + 3 * i], a1 = av[u * n3 + 3 * i + 1], a2 = av[u * n3 + 3 * i + 2];
            const double d0 = bx[3 * i], d1 = bx[3 * i + 1], d2 = bx[3 * i + 2];
            g[0] += a0;
            g[1] += a1;
            g[2] += a2;
            g[3] += d1 * a2 - d2 * a1;
            g[4] += d2 * a0 - d0 * a2;
            g[5] += d0 * a1 - d1 * a0;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) g[k] = warp_sum(g[k]);
        if (lane == 0) {
            const double* N = Nt + 36 * t;
            for (int a = 0; a < 6; ++a) {
                double acc = 0.0;
                for (int k = 0; k < 6; ++k) acc += N[6 * a + k] * (misc[16 * u + k] + g[k]);
                misc[16 * u + 8 + a] = -acc;
            }
        }
    }
    __syncthreads();
    const double* Gtt = Gt + 18LL * tmpl_off[t];   // 3n x 6
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
        const int u = e / n, b = e - u * n;
        const int p = bodies[it.y + u];
        double lb[3];
        for (int a = 0; a < 3; ++a) {
            const int row = 3 * b + a;
            double acc = av[u * n3 + row];
            for (int k = 0; k < 6; ++k) acc = fma(Gtt[6LL * row + k], misc[16 * u + 8 + k], acc);
            lb[a] = acc;
        }
        double w[3];
        rot(Rb + 9 * p, lb, w);
        const long long o = blob_gm[body_blob_off[p] + b];
        zout[o] = w[0];
        zout[o + 1] = w[1];
        zout[o + 2] = w[2];
    }
    for (int u = threadIdx.x; u < cnt; u += blockDim.x) {
        const int p = bodies[it.y + u];
        double w[3];
        const long long o = body_gm[p];
        rot(Rb + 9 * p, misc + 16 * u + 8, w);
        zout[o] = w[0];
        zout[o + 1] = w[1];
        zout[o + 2] = w[2];
        rot(Rb + 9 * p, misc + 16 * u + 11, w);
        zout[o + 3] = w[0];
        zout[o + 4] = w[1];
        zout[o + 5] = w[2];
    }
}

void launch_precond(gdc_ctx* c, const double* r, double* z, bool fp32) {
    const size_t smem = (size_t)(3 * 3 * c->max_body_blobs + 32) * sizeof(double);
    if (c->p.wall)
        ++c->n_launch, k_precond<true><<<c->NB, 128, smem, c->stream>>>(
            c->body_blob_off, c->body_tmpl, c->tmpl_n, c->tmpl_off, c->minv_off, c->blk_Minv, nullptr, c->blk_G, c->blk_N,
            c->tmpl_xyz, c->blob_gm, c->body_gm, c->Rb, r, z, c->blk_off, c->r, c->Yc);
    else if (c->tb_use && fp32)   // many bodies: grouped by template
        ++c->n_launch, k_precond_tb<true><<<c->tb_n_items, 128, c->tb_precond_smem, c->stream>>>(
            c->tb_items, c->tb_bodies, c->body_blob_off, c->tmpl_n, c->tmpl_off, c->minv_off, c->tmpl_Minv,
            c->tmpl_Minv32, c->tmpl_G, c->tmpl_N, c->tmpl_xyz, c->blob_gm, c->body_gm, c->Rb, r, z);
    else if (c->tb_use)
        ++c->n_launch, k_precond_tb<false><<<c->tb_n_items, 128, c->tb_precond_smem, c->stream>>>(
            c->tb_items, c->tb_bodies, c->body_blob_off, c->tmpl_n, c->tmpl_off, c->minv_off, c->tmpl_Minv,
            c->tmpl_Minv32, c->tmpl_G, c->tmpl_N, c->tmpl_xyz, c->blob_gm, c->body_gm, c->Rb, r, z);
    else if (fp32)
        ++c->n_launch, k_precond<false, true><<<c->NB, 128, smem, c->stream>>>(
            c->body_blob_off, c->body_tmpl, c->tmpl_n, c->tmpl_off, c->minv_off, c->tmpl_Minv, c->tmpl_Minv32, c->tmpl_G,
            c->tmpl_N, c->tmpl_xyz, c->blob_gm, c->body_gm, c->Rb, r, z, nullptr, nullptr, nullptr);
    else
        ++c->n_launch, k_precond<false><<<c->NB, 128, smem, c->stream>>>(
            c->body_blob_off, c->body_tmpl, c->tmpl_n, c->tmpl_off, c->minv_off, c->tmpl_Minv, nullptr, c->tmpl_G,
            c->tmpl_N, c->tmpl_xyz, c->blob_gm, c->body_gm, c->Rb, r, z, nullptr, nullptr, nullptr);
}

// ---- factors of the body blocks: block-preconditioned Lanczos (Sec. 4.1, Chow & Saad) ----
//
// With L_t the Cholesky factor of the template block (M_t = L_t L_t^T), L_p = R-hat_p L_t
// factors body p's block of M (M_pp = R-hat_p M_t R-hat_p^T), and the Lanczos operator of
// Chow & Saad is A = L^-1 M L^-T with L = diag_p(L_p):
//   TRI_LINV_T: out_p = L_p^-T x_p = R-hat_p (L_t^-T x_p)
//   TRI_LINV:   out_p = L_p^-1 x_p (+ add_p) = L_t^-1 (R-hat_p^T x_p) (+ add_p)
//   TRI_L:      out_p = L_p x_p = R-hat_p (L_t x_p)
// F is the template's factor stored so that out_i = sum_k F[k n3 + i] in_k (coalesced over
// the rows i); the triangular structure limits k to [i, n3) (TRI_LINV_T) or [0, i].  FP64.
// One block per body; x, add and out hold 3 doubles per blob.  Shared memory: 2 x 3n doubles.
// LAB (blobs above a wall): body p's own factor of its lab-frame block (L_p from
// k_wall_blocks, at blk_off[p]), no rotation.  T: the type of the factor and of the sums
// (float for the FP32 products of the FP32-mixed Lanczos, whose other terms carry FP32
// rounding; the rotations and the added vector stay FP64).
template <int MODE, bool LAB, typename T>
__global__ void __launch_bounds__(128) k_body_tri(const long long* __restrict__ body_blob_off,
                                                  const int* __restrict__ body_tmpl, const int* __restrict__ tmpl_n,
                                                  const long long* __restrict__ minv_off, const T* __restrict__ F,
                                                  const double* __restrict__ Rb, const double* __restrict__ x,
                                                  const double* __restrict__ add, double* __restrict__ out) {
    extern __shared__ double sh[];
    const int p = blockIdx.x;
    const int t = LAB ? p : body_tmpl[p];
    const int n = LAB ? (int)(body_blob_off[p + 1] - body_blob_off[p]) : tmpl_n[t], n3 = 3 * n;
    double* res = sh;
    T* in = reinterpret_cast<T*>(sh + n3);
    const double ident[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    const double* R = LAB ? ident : Rb + 9 * p;
    const long long i0 = body_blob_off[p];
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        double v[3] = {x[3 * (i0 + b)], x[3 * (i0 + b) + 1], x[3 * (i0 + b) + 2]};
        if (MODE == TRI_LINV) {
            double w[3];
            rotT(R, v, w);
            v[0] = w[0];
            v[1] = w[1];
            v[2] = w[2];
        }
        in[3 * b] = (T)v[0];
        in[3 * b + 1] = (T)v[1];
        in[3 * b + 2] = (T)v[2];
    }
    __syncthreads();
    const T* Ft = F + minv_off[t];
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int k0 = MODE == TRI_LINV_T ? i : 0, k1 = MODE == TRI_LINV_T ? n3 : i + 1;
        T a0 = T(0), a1 = T(0);
        int k = k0;
        for (; k + 1 < k1; k += 2) {
            a0 = fma(Ft[(long long)k * n3 + i], in[k], a0);
            a1 = fma(Ft[(long long)(k + 1) * n3 + i], in[k + 1], a1);
        }
        if (k < k1) a0 = fma(Ft[(long long)k * n3 + i], in[k], a0);
        res[i] = (double)a0 + (double)a1;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        double w[3] = {res[3 * b], res[3 * b + 1], res[3 * b + 2]};
        if (MODE != TRI_LINV) {
            double v[3];
            rot(R, w, v);
            w[0] = v[0];
            w[1] = v[1];
            w[2] = v[2];
        }
        const long long o = 3 * (i0 + b);
        if (add) {
            w[0] += add[o];
            w[1] += add[o + 1];
            w[2] += add[o + 2];
        }
        out[o] = w[0];
        out[o + 1] = w[1];
        out[o + 2] = w[2];
    }
}

// The same products for several bodies of one template per block (the bodies of item
// (t, first, count) in `bodies`): each element of the template's factor, read once from L2,
// serves all of them, where a block per body re-reads the factor body after body (at 36,121
// bodies that is hundreds of MB per launch).  One accumulator per body and row.
template <int MODE, typename T>
__global__ void __launch_bounds__(128) k_body_tri_tb(const int4* __restrict__ items, const int* __restrict__ bodies,
                                                     const long long* __restrict__ body_blob_off,
                                                     const int* __restrict__ tmpl_n,
                                                     const long long* __restrict__ minv_off, const T* __restrict__ F,
                                                     const double* __restrict__ Rb, const double* __restrict__ x,
                                                     const double* __restrict__ add, double* __restrict__ out) {
    extern __shared__ double sh[];
    const int4 it = items[blockIdx.x];
    const int t = it.x, cnt = it.z;
    const int n = tmpl_n[t], n3 = 3 * n;
    double* res = sh;                                    // [cnt][n3]
    T* in = reinterpret_cast<T*>(sh + (long long)cnt * n3);   // [cnt][n3]
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
        const int u = e / n, b = e - u * n;
        const int p = bodies[it.y + u];
        const long long o = 3 * (body_blob_off[p] + b);
        double v[3] = {x[o], x[o + 1], x[o + 2]};
        if (MODE == TRI_LINV) {
            double w[3];
            rotT(Rb + 9 * p, v, w);
            v[0] = w[0];
            v[1] = w[1];
            v[2] = w[2];
        }
        in[u * n3 + 3 * b] = (T)v[0];
        in[u * n3 + 3 * b + 1] = (T)v[1];
        in[u * n3 + 3 * b + 2] = (T)v[2];
    }
    __syncthreads();
    const T* Ft = F + minv_off[t];
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int k0 = MODE == TRI_LINV_T ? i : 0, k1 = MODE == TRI_LINV_T ? n3 : i + 1;
        T a[GDC_TB_MAX];
#pragma unroll
        for (int u = 0; u < GDC_TB_MAX; ++u) a[u] = T(0);
        for (int k = k0; k < k1; ++k) {
            const T f = Ft[(long long)k * n3 + i];
#pragma unroll
            for (int u = 0; u < GDC_TB_MAX; ++u)
                if (u < cnt) a[u] = fma(f, in[u * n3 + k], a[u]);
        }
#pragma unroll
        for (int u = 0; u < GDC_TB_MAX; ++u)
            if (u < cnt) res[u * n3 + i] = (double)a[u];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
        const int u = e / n, b = e - u * n;
        const int p = bodies[it.y + u];
        double w[3] = {res[u * n3 + 3 * b], res[u * n3 + 3 * b + 1], res[u * n3 + 3 * b + 2]};
        if (MODE != TRI_LINV) {
            double v[3];
            rot(Rb + 9 * p, w, v);
            w[0] = v[0];
            w[1] = v[1];
            w[2] = v[2];
        }
        const long long o = 3 * (body_blob_off[p] + b);
        if (add) {
            w[0] += add[o];
            w[1] += add[o + 1];
            w[2] += add[o + 2];
        }
        out[o] = w[0];
        out[o + 1] = w[1];
        out[o + 2] = w[2];
    }
}

void launch_body_tri(gdc_ctx* c, int mode, const double* x, const double* add, double* out, bool fp32) {
    const size_t smem = (size_t)(2 * 3 * c->max_body_blobs) * sizeof(double);
    const bool lab = c->p.wall != 0;
    const long long* off = lab ? c->blk_off : c->minv_off;
    // lab-frame factors (above a wall) and fewer bodies: one block per body; many bodies:
    // grouped by template
#define GDC_TRI(MODE, LAB, T, F)                                                                                  \
    do {                                                                                                          \
        if (LAB || !c->tb_use)                                                                                    \
            k_body_tri<MODE, LAB, T><<<c->NB, 128, smem, c->stream>>>(c->body_blob_off, c->body_tmpl, c->tmpl_n,  \
                                                                     off, F, c->Rb, x, add, out);                \
        else                                                                                                      \
            k_body_tri_tb<MODE, T><<<c->tb_n_items, 128, c->tb_smem, c->stream>>>(                               \
                c->tb_items, c->tb_bodies, c->body_blob_off, c->tmpl_n, c->minv_off, F, c->Rb, x, add, out);     \
    } while (0)
    ++c->n_launch;
    if (fp32 && !lab && mode == TRI_LINV_T)
        GDC_TRI(TRI_LINV_T, false, float, c->tmpl_X32);
    else if (fp32 && !lab && mode == TRI_LINV)
        GDC_TRI(TRI_LINV, false, float, c->tmpl_XT32);
    else if (mode == TRI_LINV_T) {
        if (lab) GDC_TRI(TRI_LINV_T, true, double, c->blk_X); else GDC_TRI(TRI_LINV_T, false, double, c->tmpl_X);
    } else if (mode == TRI_LINV) {
        if (lab) GDC_TRI(TRI_LINV, true, double, c->blk_XT); else GDC_TRI(TRI_LINV, false, double, c->tmpl_XT);
    } else {
        if (lab) GDC_TRI(TRI_L, true, double, c->blk_LT); else GDC_TRI(TRI_L, false, double, c->tmpl_LT);
    }
#undef GDC_TRI
}

// ---- per-template setup (once, at init) -------------------------------------------------

// Cyclic Jacobi eigendecomposition of a symmetric 6x6 (Golub & Van Loan, Sec. 8.5), then the
// pseudo-inverse with eigenvalues below rel_tol * max set to zero.  Single thread.
__device__ void pinv6(const double* A_in, double* P, double rel_tol) {
    double A[36], V[36];
    for (int k = 0; k < 36; ++k) {
        A[k] = A_in[k];
        V[k] = (k % 7 == 0) ? 1.0 : 0.0;
    }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                tot += A[6 * i + j] * A[6 * i + j];
                if (i != j) off += A[6 * i + j] * A[6 * i + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int pp = 0; pp < 5; ++pp)
            for (int qq = pp + 1; qq < 6; ++qq) {
                const double apq = A[6 * pp + qq];
                if (apq == 0.0) continue;
                const double tau = (A[6 * qq + qq] - A[6 * pp + pp]) / (2.0 * apq);
                const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = tt * cs;
                // A <- J^T A J, J = identity with [c s; -s c] in rows/cols (pp, qq)
                for (int k = 0; k < 6; ++k) {
                    const double akp = A[6 * k + pp], akq = A[6 * k + qq];
                    A[6 * k + pp] = cs * akp - sn * akq;
                    A[6 * k + qq] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 6; ++k) {
                    const double apk = A[6 * pp + k], aqk = A[6 * qq + k];
                    A[6 * pp + k] = cs * apk - sn * aqk;
                    A[6 * qq + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 6; ++k) {
                    const double vkp = V[6 * k + pp], vkq = V[6 * k + qq];
                    V[6 * k + pp] = cs * vkp - sn * vkq;
                    V[6 * k + qq] = sn * vkp + cs * vkq;
                }
            }
    }
    double lmax = 0.0;
    for (int i = 0; i < 6; ++i) lmax = fmax(lmax, fabs(A[7 * i]));
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 6; ++k) {
                const double lam = A[7 * k];
                if (lam > rel_tol * lmax) acc += V[6 * i + k] * V[6 * j + k] / lam;
            }
            P[6 * i + j] = acc;
        }
}

// One block per template.  work: 2 (3n)^2 doubles of scratch per template at minv_off.
__global__ void k_template_setup(const int* __restrict__ tmpl_n, const int* __restrict__ tmpl_off,
                                 const long long* __restrict__ minv_off, const double* __restrict__ xyz,
                                 double a, double eta, double* __restrict__ Minv, double* __restrict__ Gt,
                                 double* __restrict__ Nt, double* __restrict__ KtKp, double* __restrict__ work,
                                 double* __restrict__ Mt, const double* __restrict__ Mext, int* __restrict__ status,
                                 double* __restrict__ LT, double* __restrict__ Xo, double* __restrict__ XT) {
    const int t = blockIdx.x;
    const int n = tmpl_n[t];
    const int n3 = 3 * n;
    const double* b = xyz + 3LL * tmpl_off[t];
    double* Mi = Minv + minv_off[t];
    double* L = work + 2 * minv_off[t];
    double* X = L + (long long)n3 * n3;
    const double c0 = 1.0 / (8.0 * 3.141592653589793 * eta);
    // 1. the template's mobility block M_t, row-major in L: given (Mext: the FCM block of the
    //    template alone in the periodic cube), or the RPY block (Sec. 4.1)
    for (long long e = threadIdx.x; Mext && e < (long long)n3 * n3; e += blockDim.x) {
        L[e] = Mext[minv_off[t] + e];
        Mt[minv_off[t] + e] = L[e];
    }
    for (long long e = threadIdx.x; !Mext && e < (long long)n3 * n3; e += blockDim.x) {
        const int row = (int)(e / n3), col = (int)(e % n3);
        const int i = row / 3, al = row % 3, j = col / 3, be = col % 3;
        const double d0 = b[3 * j] - b[3 * i], d1 = b[3 * j + 1] - b[3 * i + 1], d2 = b[3 * j + 2] - b[3 * i + 2];
        const double dd[3] = {d0, d1, d2};
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        double A, B;
        if (r2 == 0.0) {
            A = 4.0 / (3.0 * a);
            B = 0.0;
        } else if (r2 < 4.0 * a * a) {
            const double r = sqrt(r2);
            A = 4.0 / (3.0 * a) * (1.0 - 9.0 * r / (32.0 * a));
            B = 1.0 / (8.0 * a * a * r);
        } else {
            const double r = sqrt(r2);
            A = 1.0 / r + 2.0 * a * a / (3.0 * r * r2);
            B = (1.0 - 2.0 * a * a / r2) / (r * r2);
        }
        L[e] = c0 * ((al == be ? A : 0.0) + B * dd[al] * dd[be]);
        Mt[minv_off[t] + e] = L[e];
    }
    __syncthreads();
    // 2. Cholesky M = L L^T (right-looking; lower triangle of L overwritten)
    for (int k = 0; k < n3; ++k) {
        if (threadIdx.x == 0) {
            const double dkk = L[(long long)k * n3 + k];
            if (!(dkk > 0.0)) atomicExch(status, 1);
            L[(long long)k * n3 + k] = sqrt(fmax(dkk, 1e-300));
        }
        __syncthreads();
        const double lkk = L[(long long)k * n3 + k];
        for (int i = k + 1 + threadIdx.x; i < n3; i += blockDim.x) L[(long long)i * n3 + k] /= lkk;
        __syncthreads();
        const int m = n3 - k - 1;
        for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
            const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
            if (j <= i) L[(long long)i * n3 + j] -= L[(long long)i * n3 + k] * L[(long long)j * n3 + k];
        }
        __syncthreads();
    }
    // 3. X = L^-1 column by column (forward substitution), then M^-1 = X^T X
    for (int col = threadIdx.x; col < n3; col += blockDim.x) {
        for (int i = 0; i < n3; ++i) X[(long long)i * n3 + col] = 0.0;
        for (int i = col; i < n3; ++i) {
            double acc = (i == col) ? 1.0 : 0.0;
            for (int k = col; k < i; ++k) acc -= L[(long long)i * n3 + k] * X[(long long)k * n3 + col];
            X[(long long)i * n3 + col] = acc / L[(long long)i * n3 + i];
        }
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)n3 * n3; e += blockDim.x) {
        const int i = (int)(e / n3), j = (int)(e % n3);
        double acc = 0.0;
        for (int k = max(i, j); k < n3; ++k) acc += X[(long long)k * n3 + i] * X[(long long)k * n3 + j];
        Mi[e] = acc;
        // the factors for the preconditioned Lanczos operator (L lower; its upper part still
        // holds M and is not part of the factor; X = L^-1 is lower with zeros above)
        const long long o = minv_off[t] + e;
        LT[o] = j >= i ? L[(long long)j * n3 + i] : 0.0;
        Xo[o] = X[e];
        XT[o] = X[(long long)j * n3 + i];
    }
    __syncthreads();
    // 4. G = M^-1 K_t (3n x 6): K_t columns are unit translations and rotations e_b x b_i
    double* G = Gt + 18LL * tmpl_off[t];
    for (long long e = threadIdx.x; e < 6LL * n3; e += blockDim.x) {
        const int row = (int)(e / 6), col = (int)(e % 6);
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            double kc[3];
            if (col < 3) {
                kc[0] = col == 0;
                kc[1] = col == 1;
                kc[2] = col == 2;
            } else {
                const int bb = col - 3;  // e_bb x b_i
                const double e3[3] = {(double)(bb == 0), (double)(bb == 1), (double)(bb == 2)};
                kc[0] = e3[1] * b[3 * i + 2] - e3[2] * b[3 * i + 1];
                kc[1] = e3[2] * b[3 * i] - e3[0] * b[3 * i + 2];
                kc[2] = e3[0] * b[3 * i + 1] - e3[1] * b[3 * i];
            }
            for (int al = 0; al < 3; ++al) acc += Mi[(long long)row * n3 + 3 * i + al] * kc[al];
        }
        G[e] = acc;
    }
    __syncthreads();
    // 5. N_t = (K_t^T G)^+ and (K_t^T K_t)^+  (closed form of Sec. 5 for the latter)
    if (threadIdx.x == 0) {
        double A6[36], KK[36];
        for (int k = 0; k < 36; ++k) {
            A6[k] = 0.0;
            KK[k] = 0.0;
        }
        for (int i = 0; i < n; ++i) {
            const double bx = b[3 * i], by = b[3 * i + 1], bz = b[3 * i + 2];
            // K_i = [I, [x b]]: columns e_x, e_y, e_z and e_k x b_i
            double Kc[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, -bz, by}, {bz, 0, -bx}, {-by, bx, 0}};
            for (int u = 0; u < 6; ++u)
                for (int v = 0; v < 6; ++v) {
                    double s1 = 0.0, s2 = 0.0;
                    for (int al = 0; al < 3; ++al) {
                        s1 += Kc[u][al] * G[6LL * (3 * i + al) + v];
                        s2 += Kc[u][al] * Kc[v][al];
                    }
                    A6[6 * u + v] += s1;
                    KK[6 * u + v] += s2;
                }
        }
        for (int u = 0; u < 6; ++u)  // symmetrise rounding
            for (int v = u + 1; v < 6; ++v) {
                const double m = 0.5 * (A6[6 * u + v] + A6[6 * v + u]);
                A6[6 * u + v] = A6[6 * v + u] = m;
            }
        pinv6(A6, Nt + 36 * t, 1e-10);
        pinv6(KK, KtKp + 36 * t, 1e-10);
    }
}

void launch_template_setup(gdc_ctx* c, const double* Mext) {
    ++c->n_launch, k_template_setup<<<c->T, 256, 0, c->stream>>>(c->tmpl_n, c->tmpl_off, c->minv_off, c->tmpl_xyz, c->p.a, c->p.eta,
                                                  c->tmpl_Minv, c->tmpl_G, c->tmpl_N, c->tmpl_KtKp, c->tmpl_work,
                                                  c->tmpl_M, Mext, c->dev_status, c->tmpl_LT, c->tmpl_X, c->tmpl_XT);
    const long long nm = c->h_minv_off[c->T];
    const int gr = (int)std::min<long long>(ceil_div(nm, 256), 1024);
    ++c->n_launch, k_round_f32<<<gr, 256, 0, c->stream>>>(nm, c->tmpl_M, c->tmpl_M32);
    ++c->n_launch, k_round_f32<<<gr, 256, 0, c->stream>>>(nm, c->tmpl_X, c->tmpl_X32);
    ++c->n_launch, k_round_f32<<<gr, 256, 0, c->stream>>>(nm, c->tmpl_Minv, c->tmpl_Minv32);
    ++c->n_launch, k_round_f32<<<gr, 256, 0, c->stream>>>(nm, c->tmpl_XT, c->tmpl_XT32);
}

// ---- per-body blocks above a wall (Sec. 4.1, Sec. 6.2) ---------------------------------
//
// A wall makes a body's block of M depend on its height and orientation, so the blocks of
// the preconditioner (the exact per-body saddle solve) and the factors of the
// preconditioned Lanczos operator are set up for every body at every configuration.  One
// block per body: M_pp = unbounded RPY + wall correction (wall_pair.cuh) from the blob
// offsets d_i = r_i - Y_p and the heights, in FP64; its Cholesky factor L, X = L^-1,
// M_pp^-1 = X^T X, G = M_pp^-1 K_p (K_p from d), N = (K_p^T G)^+, and LT = L^T, X, XT = X^T
// stored for k_body_tri<LAB>.  A blob at or below z = a (overlapping the wall, where the
// correction is not a mobility) sets status[2]; a block that is not positive definite sets
// status[0] = 1.  Shared memory: 3n doubles.
__global__ void __launch_bounds__(256) k_wall_blocks(const long long* __restrict__ body_blob_off,
                                                     const long long* __restrict__ blk_off, const double* __restrict__ r,
                                                     const double* __restrict__ Yc, double a, double eta,
                                                     double* __restrict__ work, double* __restrict__ Minv,
                                                     double* __restrict__ Gb, double* __restrict__ Nb,
                                                     double* __restrict__ LT, double* __restrict__ Xo,
                                                     double* __restrict__ XT, int* __restrict__ status) {
    extern __shared__ double dsh[];
    const int p = blockIdx.x;
    const long long i0 = body_blob_off[p];
    const int n = (int)(body_blob_off[p + 1] - i0), n3 = 3 * n;
    double* d = dsh;
    const double zc = Yc[3 * p + 2];
    for (int e = threadIdx.x; e < n3; e += blockDim.x) d[e] = r[3 * i0 + e] - Yc[3 * p + e % 3];
    for (int b = threadIdx.x; b < n; b += blockDim.x)
        if (!(r[3 * (i0 + b) + 2] > a)) atomicExch(status + 2, 1);
    __syncthreads();
    const long long mo = blk_off[p];
    double* L = work + 2 * mo;
    double* X = L + (long long)n3 * n3;
    const double c0 = 1.0 / (8.0 * 3.141592653589793 * eta);
    // 1. M_pp row-major in L: RPY entry (units of 1/(8 pi eta)) + wall correction of column be
    for (long long e = threadIdx.x; e < (long long)n3 * n3; e += blockDim.x) {
        const int row = (int)(e / n3), col = (int)(e % n3);
        const int i = row / 3, al = row % 3, j = col / 3, be = col % 3;
        const double dx = d[3 * j] - d[3 * i], dy = d[3 * j + 1] - d[3 * i + 1], dz = d[3 * j + 2] - d[3 * i + 2];
        const double dd[3] = {dx, dy, dz};
        const double r2 = dx * dx + dy * dy + dz * dz;
        double A, B;
        if (r2 == 0.0) {
            A = 4.0 / (3.0 * a);
            B = 0.0;
        } else if (r2 < 4.0 * a * a) {
            const double rr = sqrt(r2);
            A = 4.0 / (3.0 * a) * (1.0 - 9.0 * rr / (32.0 * a));
            B = 1.0 / (8.0 * a * a * rr);
        } else {
            const double rr = sqrt(r2);
            A = 1.0 / rr + 2.0 * a * a / (3.0 * rr * r2);
            B = (1.0 - 2.0 * a * a / r2) / (rr * r2);
        }
        double w[3] = {0.0, 0.0, 0.0};
        wall_pair<double>(d[3 * i] - d[3 * j], d[3 * i + 1] - d[3 * j + 1], d[3 * i + 2] + d[3 * j + 2] + 2.0 * zc,
                          d[3 * j + 2] + zc, a * a, be == 0 ? 1.0 : 0.0, be == 1 ? 1.0 : 0.0, be == 2 ? 1.0 : 0.0,
                          w[0], w[1], w[2]);
        L[e] = c0 * ((al == be ? A : 0.0) + B * dd[al] * dd[be] + w[al]);
    }
    __syncthreads();
    // 2. Cholesky M = L L^T (right-looking; lower triangle of L overwritten)
    for (int k = 0; k < n3; ++k) {
        if (threadIdx.x == 0) {
            const double dkk = L[(long long)k * n3 + k];
            if (!(dkk > 0.0)) atomicExch(status, 1);
            L[(long long)k * n3 + k] = sqrt(fmax(dkk, 1e-300));
        }
        __syncthreads();
        const double lkk = L[(long long)k * n3 + k];
        for (int i = k + 1 + threadIdx.x; i < n3; i += blockDim.x) L[(long long)i * n3 + k] /= lkk;
        __syncthreads();
        const int m = n3 - k - 1;
        for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
            const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
            if (j <= i) L[(long long)i * n3 + j] -= L[(long long)i * n3 + k] * L[(long long)j * n3 + k];
        }
        __syncthreads();
    }
    // 3. X = L^-1 (forward substitution per column), M^-1 = X^T X and the factor layouts
    for (int col = threadIdx.x; col < n3; col += blockDim.x) {
        for (int i = 0; i < n3; ++i) X[(long long)i * n3 + col] = 0.0;
        for (int i = col; i < n3; ++i) {
            double acc = (i == col) ? 1.0 : 0.0;
            for (int k = col; k < i; ++k) acc -= L[(long long)i * n3 + k] * X[(long long)k * n3 + col];
            X[(long long)i * n3 + col] = acc / L[(long long)i * n3 + i];
        }
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)n3 * n3; e += blockDim.x) {
        const int i = (int)(e / n3), j = (int)(e % n3);
        double acc = 0.0;
        for (int k = max(i, j); k < n3; ++k) acc += X[(long long)k * n3 + i] * X[(long long)k * n3 + j];
        Minv[mo + e] = acc;
        LT[mo + e] = j >= i ? L[(long long)j * n3 + i] : 0.0;
        Xo[mo + e] = X[e];
        XT[mo + e] = X[(long long)j * n3 + i];
    }
    __syncthreads();
    // 4. G = M^-1 K (3n x 6), K columns: unit translations and e_c x d_i
    double* G = Gb + 18LL * i0;
    for (long long e = threadIdx.x; e < 6LL * n3; e += blockDim.x) {
        const int row = (int)(e / 6), col = (int)(e % 6);
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            double kc[3];
            if (col < 3) {
                kc[0] = col == 0;
                kc[1] = col == 1;
                kc[2] = col == 2;
            } else {
                const int bb = col - 3;
                const double e3[3] = {(double)(bb == 0), (double)(bb == 1), (double)(bb == 2)};
                kc[0] = e3[1] * d[3 * i + 2] - e3[2] * d[3 * i + 1];
                kc[1] = e3[2] * d[3 * i] - e3[0] * d[3 * i + 2];
                kc[2] = e3[0] * d[3 * i + 1] - e3[1] * d[3 * i];
            }
            for (int al = 0; al < 3; ++al) acc += Minv[mo + (long long)row * n3 + 3 * i + al] * kc[al];
        }
        G[e] = acc;
    }
    __syncthreads();
    // 5. N = (K^T G)^+ (symmetrised, pseudo-inverse for collinear bodies)
    if (threadIdx.x == 0) {
        double A6[36];
        for (int k = 0; k < 36; ++k) A6[k] = 0.0;
        for (int i = 0; i < n; ++i) {
            const double bx = d[3 * i], by = d[3 * i + 1], bz = d[3 * i + 2];
            double Kc[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, -bz, by}, {bz, 0, -bx}, {-by, bx, 0}};
            for (int u = 0; u < 6; ++u)
                for (int v = 0; v < 6; ++v) {
                    double s1 = 0.0;
                    for (int al = 0; al < 3; ++al) s1 += Kc[u][al] * G[6LL * (3 * i + al) + v];
                    A6[6 * u + v] += s1;
                }
        }
        for (int u = 0; u < 6; ++u)
            for (int v = u + 1; v < 6; ++v) {
                const double m = 0.5 * (A6[6 * u + v] + A6[6 * v + u]);
                A6[6 * u + v] = A6[6 * v + u] = m;
            }
        pinv6(A6, Nb + 36LL * p, 1e-10);
    }
}

void launch_wall_blocks(gdc_ctx* c) {
    ++c->n_launch, k_wall_blocks<<<c->NB, 256, (size_t)3 * c->max_body_blobs * sizeof(double), c->stream>>>(
        c->body_blob_off, c->blk_off, c->r, c->Yc, c->p.a, c->p.eta, c->blk_work, c->blk_Minv, c->blk_G, c->blk_N,
        c->blk_LT, c->blk_X, c->blk_XT, c->dev_status);
}

}  // namespace gdc
