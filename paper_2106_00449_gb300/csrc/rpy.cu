// On-the-fly tiled N-body kernels: the RPY product u = M lambda (Sec. 4.1, Eq. ddof_mob) in
// FP32 and FP64, and the soft blob repulsion (Eq. soft_sphere_potential form).  Sources are staged in
// shared memory tile by tile; each thread owns TPT targets.  Work is split into
// (target tile x source chunk) items so that a launch fills every SM several times
// over; chunk partial sums are added in FP64, in chunk order, by the epilogue.
//
// RPY with c0 = 1/(8 pi eta), d = r_j - r_i, r = |d| (the d d^T term is even in d):
//   r >= 2a : u_i += c0 [ (1/r + 2a^2/(3 r^3)) lambda_j + (1/r^3)(1 - 2a^2/r^2) (d.lambda_j) d ]
//   r <  2a : u_i += c0 [ (4/(3a))(1 - 9r/(32a)) lambda_j + (1/(8 a^2 r)) (d.lambda_j) d ]
//   r == 0  : u_i += c0 (4/(3a)) lambda_j                     (self term 1/(6 pi eta a))
#include <algorithm>
#include <numeric>

#include "common.cuh"
#include "pair_common.cuh"
#include "df.cuh"
#include "forces.cuh"

namespace gdc {

#ifndef GDC_MV_TILE
#define GDC_MV_TILE 256
#endif
constexpr int MV_TILE = GDC_MV_TILE;   // sources staged in shared memory per tile

// ---- source packing ---------------------------------------------------------

// FP32 sources in the layout the pair kernel's shared-memory tiles use, three float4 per
// blob: (x,x,y,y) (z,z,lx,lx) (ly,ly,lz,lz) -- each value twice, one per packed lane.
__global__ void k_pack_lam32(int NBL, const int* __restrict__ map, const double* __restrict__ x,
                             const float4* __restrict__ spos, float4* __restrict__ sdup) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const long long o = map ? (long long)map[i] : 3LL * i;
    const float lx = (float)x[o], ly = (float)x[o + 1], lz = (float)x[o + 2];
    const float4 ps = spos[i];
    sdup[3 * i] = make_float4(ps.x, ps.x, ps.y, ps.y);
    sdup[3 * i + 1] = make_float4(ps.z, ps.z, lx, lx);
    sdup[3 * i + 2] = make_float4(ly, ly, lz, lz);
}

__global__ void k_pack_lam64(int NBL, const int* __restrict__ map, const double* __restrict__ x,
                             double4_32a* __restrict__ slam) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const long long o = map ? (long long)map[i] : 3LL * i;
    slam[i] = make_double4_32a(x[o], x[o + 1], x[o + 2], 0.0);
}

void launch_pack_lambda(gdc_ctx* c, int prec, const double* x, int gm_layout) {
    const int* map = gm_layout ? c->blob_gm : nullptr;
    if (prec == GDC_FP32_MIXED)
        ++c->n_launch, k_pack_lam32<<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(c->NBL, map, x, c->spos, c->sdup);
    else
        ++c->n_launch, k_pack_lam64<<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(c->NBL, map, x, c->slam64);
}

// ---- FP32 RPY pair kernel -----------------------------------------------------

// Each thread owns 2P targets, evaluated two at a time with packed instructions.  Every
// pair of the suspension is evaluated with the far-field form of the RPY tensor at the
// clamped distance max(r, 2a) (branch free); the self pair and the pairs closer than 2a,
// for which that is not the RPY tensor, are corrected in FP64 by the epilogue from a list of
// such pairs built once per configuration.  Shared memory holds each source as
// (x,x,y,y) (z,z,lx,lx) (ly,ly,lz,lz), so one 16-byte load feeds a packed operand.  Sums run
// over 32-source sub-chunks, then per tile, then across tiles with compensation.
//
// Source tiles are staged by the bulk-copy (TMA) engine: the packed source array already
// holds the duplicated layout, so a tile is one contiguous cp.async.bulk into shared
// memory, completed on an mbarrier.  Two buffers: the copy of tile t+1 runs while tile t
// is evaluated.  Waits are bounded; on a timeout the kernel flags status[1] and returns.

// MINB: resident blocks per SM the register allocator is asked to allow, 4 (112 / 124
// registers for P = 1 / 2) or 6 (76 / 80, the latter with a few spilled bytes); the
// autotuner times both.
template <int P, int MINB>
__global__ void __launch_bounds__(128, MINB) k_rpy32(const MvItem* __restrict__ items, const int* __restrict__ active,
                                               const long long* __restrict__ susp_blob_off,
                                               const float4* __restrict__ spos, const float4* __restrict__ sdup,
                                               float4* __restrict__ part, int NBL, RpyConst32 k,
                                               int* __restrict__ status, int first_polls) {
    __shared__ __align__(128) float4 shbuf[2][3 * MV_TILE];
    __shared__ __align__(8) unsigned long long mbar[2];
    const MvItem it = items[blockIdx.x];
    const long long b0 = susp_blob_off[it.s];
    const int ns = (int)(susp_blob_off[it.s + 1] - b0);
    if (active && !active[it.s]) {
        // a suspension whose Krylov loop has stopped: its product is not used; leave zeros
        for (int t = threadIdx.x; t < 256 * P && it.t0 + t < ns; t += 128)
            part[(long long)it.k * NBL + b0 + it.t0 + t] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float2 c23 = make_float2(k.c23, k.c23), mc2 = make_float2(-k.c2, -k.c2), one = make_float2(1.f, 1.f);
    const float four_a2 = k.four_a2;
    const int ntile = (it.j1 - it.j0 + MV_TILE - 1) / MV_TILE;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && ntile > 0)
        bulk_tile_load(shbuf[0], sdup + 3 * (b0 + it.j0), 48u * (unsigned)min(MV_TILE, it.j1 - it.j0), &mbar[0]);

    float2 xt[P], yt[P], zt[P], ax[P], ay[P], az[P], cx[P], cy[P], cz[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float4 pa = spos[b0 + min(it.t0 + (int)threadIdx.x + (2 * p) * 128, ns - 1)];
        const float4 pb = spos[b0 + min(it.t0 + (int)threadIdx.x + (2 * p + 1) * 128, ns - 1)];
        xt[p] = make_float2(pa.x, pb.x);
        yt[p] = make_float2(pa.y, pb.y);
        zt[p] = make_float2(pa.z, pb.z);
        ax[p] = ay[p] = az[p] = make_float2(0.f, 0.f);
        cx[p] = cy[p] = cz[p] = make_float2(0.f, 0.f);
    }
    for (int t = 0; t < ntile; ++t) {
        const int j0 = it.j0 + t * MV_TILE;
        const int n = min(MV_TILE, it.j1 - j0);
        const float4* sh = shbuf[t & 1];
        if (threadIdx.x == 0 && t + 1 < ntile) {
            // buffer (t+1)&1 was last read in iteration t-1, which ended with a barrier
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int j1n = j0 + MV_TILE;
            bulk_tile_load(shbuf[(t + 1) & 1], sdup + 3 * (b0 + j1n), 48u * (unsigned)min(MV_TILE, it.j1 - j1n),
                           &mbar[(t + 1) & 1]);
        }
        const bool ok = mbar_wait(&mbar[t & 1], (unsigned)((t >> 1) & 1), first_polls);
        float2 tx[P], ty[P], tz[P];
#pragma unroll
        for (int p = 0; p < P; ++p) tx[p] = ty[p] = tz[p] = make_float2(0.f, 0.f);
        for (int jc = 0; jc < n; jc += 32) {
            const int je = min(jc + 32, n);
            float2 qx[P], qy[P], qz[P];
#pragma unroll
            for (int p = 0; p < P; ++p) qx[p] = qy[p] = qz[p] = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int j = jc; j < je; ++j) {
                const float4 s0 = sh[3 * j], s1 = sh[3 * j + 1], s2 = sh[3 * j + 2];
                const float2 xs = make_float2(s0.x, s0.y), ys = make_float2(s0.z, s0.w), zs = make_float2(s1.x, s1.y);
                const float2 lx = make_float2(s1.z, s1.w), ly = make_float2(s2.x, s2.y), lz = make_float2(s2.z, s2.w);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float2 dx = sub2(xs, xt[p]), dy = sub2(ys, yt[p]), dz = sub2(zs, zt[p]);
                    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
                    const float2 ri = make_float2(rsqrtf(fmaxf(r2.x, four_a2)), rsqrtf(fmaxf(r2.y, four_a2)));
                    const float2 ri2 = mul2(ri, ri);
                    const float2 ri3 = mul2(ri2, ri);
                    const float2 A = fma2(c23, ri3, ri);
                    const float2 B = mul2(ri3, fma2(mc2, ri2, one));
                    const float2 s = mul2(B, fma2(dx, lx, fma2(dy, ly, mul2(dz, lz))));
                    qx[p] = fma2(A, lx, fma2(s, dx, qx[p]));
                    qy[p] = fma2(A, ly, fma2(s, dy, qy[p]));
                    qz[p] = fma2(A, lz, fma2(s, dz, qz[p]));
                }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                tx[p] = add2(tx[p], qx[p]);
                ty[p] = add2(ty[p], qy[p]);
                tz[p] = add2(tz[p], qz[p]);
            }
        }
        // compensated (Kahan) addition of the tile sums
#pragma unroll
        for (int p = 0; p < P; ++p) {
            float2 y, u;
            y = sub2(tx[p], cx[p]); u = add2(ax[p], y); cx[p] = sub2(sub2(u, ax[p]), y); ax[p] = u;
            y = sub2(ty[p], cy[p]); u = add2(ay[p], y); cy[p] = sub2(sub2(u, ay[p]), y); ay[p] = u;
            y = sub2(tz[p], cz[p]); u = add2(az[p], y); cz[p] = sub2(sub2(u, az[p]), y); az[p] = u;
        }
        // every thread is done with this buffer before it is refilled; a timed-out copy stops the block
        // after its copies in flight have landed: tile t's (whose wait gave up) and tile t+1's
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(status + 1, 1);
                mbar_wait(&mbar[t & 1], (unsigned)((t >> 1) & 1));
                if (t + 1 < ntile) mbar_wait(&mbar[(t + 1) & 1], (unsigned)(((t + 1) >> 1) & 1));
            }
            return;
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float2 rx = sub2(ax[p], cx[p]), ry = sub2(ay[p], cy[p]), rz = sub2(az[p], cz[p]);
        const int ta = it.t0 + threadIdx.x + (2 * p) * 128, tb = ta + 128;
        if (ta < ns) part[(long long)it.k * NBL + b0 + ta] = make_float4(rx.x, ry.x, rz.x, 0.f);
        if (tb < ns) part[(long long)it.k * NBL + b0 + tb] = make_float4(rx.y, ry.y, rz.y, 0.f);
    }
}

// ---- double-float (df64) RPY pair kernel for accurate residuals ----------------------
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so the accurate product that
// the mixed-precision mobility solve checks its residual with evaluates the pairs of
// different bodies in double-float arithmetic on the FP32 pipes: a value is an
// unevaluated sum hi + lo of two floats (about 48 significant bits).  The error-free
// transformations are Knuth's two-sum, Dekker's fast two-sum and the FMA-based exact
// product.  Same-body pairs are skipped (added exactly in FP64 by k_intra_body).

template <int TPT>
__global__ void __launch_bounds__(128) k_rpy_df(const MvItem* __restrict__ items, const long long* __restrict__ susp_blob_off,
                                                const double4_32a* __restrict__ spos, const double4_32a* __restrict__ slam,
                                                double4_32a* __restrict__ part, int NBL, RpyConstDF k) {
    __shared__ float4 sh[4 * MV_TILE];
    const MvItem it = items[blockIdx.x];
    const long long b0 = susp_blob_off[it.s];
    const int ns = (int)(susp_blob_off[it.s + 1] - b0);
    df xt[TPT], yt[TPT], zt[TPT], ux[TPT], uy[TPT], uz[TPT];
    float bt[TPT];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const double4_32a p = spos[b0 + min(it.t0 + (int)threadIdx.x + t * 128, ns - 1)];
        xt[t] = df_from(p.x);
        yt[t] = df_from(p.y);
        zt[t] = df_from(p.z);
        bt[t] = (float)p.w;
        ux[t] = uy[t] = uz[t] = df{0.f, 0.f};
    }
    const df one{1.f, 0.f};
    for (int j0 = it.j0; j0 < it.j1; j0 += MV_TILE) {
        const int n = min(MV_TILE, it.j1 - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < n; e += 128) {
            const double4_32a ps = spos[b0 + j0 + e];
            const double4_32a ls = slam[b0 + j0 + e];
            const df x = df_from(ps.x), y = df_from(ps.y), z = df_from(ps.z);
            const df lx = df_from(ls.x), ly = df_from(ls.y), lz = df_from(ls.z);
            sh[4 * e] = make_float4(x.h, y.h, z.h, (float)ps.w);
            sh[4 * e + 1] = make_float4(x.l, y.l, z.l, 0.f);
            sh[4 * e + 2] = make_float4(lx.h, ly.h, lz.h, 0.f);
            sh[4 * e + 3] = make_float4(lx.l, ly.l, lz.l, 0.f);
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const float4 s0 = sh[4 * j], s1 = sh[4 * j + 1], s2 = sh[4 * j + 2], s3 = sh[4 * j + 3];
            const df lx{s2.x, s3.x}, ly{s2.y, s3.y}, lz{s2.z, s3.z};
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                if (s0.w == bt[t]) continue;   // same body: exact FP64 block elsewhere
                const df dx = df_sub(df{s0.x, s1.x}, xt[t]);
                const df dy = df_sub(df{s0.y, s1.y}, yt[t]);
                const df dz = df_sub(df{s0.z, s1.z}, zt[t]);
                const df r2 = df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz));
                const df ri = df_rsqrt(r2);
                df A, B;
                // r^2 >= 4a^2 compared in double-float (both normalised: high parts first)
                if (r2.h > k.four_a2.h || (r2.h == k.four_a2.h && r2.l >= k.four_a2.l)) {
                    const df ri2 = df_mul(ri, ri);
                    const df ri3 = df_mul(ri2, ri);
                    A = df_add(ri, df_mul(k.c23, ri3));
                    B = df_mul(ri3, df_sub(one, df_mul(k.c2, ri2)));
                } else {   // overlapping blobs of different bodies (r > 0 for distinct blobs)
                    const df r = df_mul(r2, ri);
                    A = df_mul(k.cA, df_sub(one, df_mul(k.c9, r)));
                    B = df_mul(k.cB, ri);
                }
                const df dl = df_add(df_add(df_mul(dx, lx), df_mul(dy, ly)), df_mul(dz, lz));
                const df s = df_mul(B, dl);
                ux[t] = df_add(ux[t], df_add(df_mul(A, lx), df_mul(s, dx)));
                uy[t] = df_add(uy[t], df_add(df_mul(A, ly), df_mul(s, dy)));
                uz[t] = df_add(uz[t], df_add(df_mul(A, lz), df_mul(s, dz)));
            }
        }
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int ti = it.t0 + threadIdx.x + t * 128;
        if (ti < ns) part[(long long)it.k * NBL + b0 + ti] = make_double4_32a(df_to(ux[t]), df_to(uy[t]), df_to(uz[t]), 0.0);
    }
}

template <int TPT>
__global__ void __launch_bounds__(128) k_rpy64(const MvItem* __restrict__ items, const int* __restrict__ active,
                                               const long long* __restrict__ susp_blob_off,
                                               const double4_32a* __restrict__ spos, const double4_32a* __restrict__ slam,
                                               double4_32a* __restrict__ part, int NBL, double a) {
    __shared__ double4_32a sp[MV_TILE];
    __shared__ double4_32a sl[MV_TILE];
    const MvItem it = items[blockIdx.x];
    const long long b0 = susp_blob_off[it.s];
    const int ns = (int)(susp_blob_off[it.s + 1] - b0);
    if (active && !active[it.s]) {   // stopped Krylov loop: product unused, leave zeros
        for (int t = threadIdx.x; t < 128 * TPT && it.t0 + t < ns; t += 128)
            part[(long long)it.k * NBL + b0 + it.t0 + t] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const double c23 = 2.0 * a * a / 3.0, c2 = 2.0 * a * a, four_a2 = 4.0 * a * a;
    const double cA = 4.0 / (3.0 * a), c9 = 9.0 / (32.0 * a), cB = 1.0 / (8.0 * a * a);
    double xt[TPT], yt[TPT], zt[TPT], ax[TPT], ay[TPT], az[TPT];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int ti = it.t0 + threadIdx.x + t * 128;
        const double4_32a p = spos[b0 + min(ti, ns - 1)];
        xt[t] = p.x;
        yt[t] = p.y;
        zt[t] = p.z;
        ax[t] = ay[t] = az[t] = 0.0;
    }
    for (int j0 = it.j0; j0 < it.j1; j0 += MV_TILE) {
        const int n = min(MV_TILE, it.j1 - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < n; e += 128) {
            sp[e] = spos[b0 + j0 + e];
            sl[e] = slam[b0 + j0 + e];
        }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const double4_32a ps = sp[j];
            const double4_32a ls = sl[j];
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                const double dx = ps.x - xt[t], dy = ps.y - yt[t], dz = ps.z - zt[t];
                const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                double A, B;
                if (r2 < four_a2) {
                    if (r2 > 0.0) {
                        const double r = sqrt(r2);
                        A = cA * fma(-c9, r, 1.0);
                        B = cB / r;
                    } else {
                        A = cA;
                        B = 0.0;
                    }
                } else {
                    const double ri = rsqrt(r2);
                    const double ri2 = ri * ri, ri3 = ri2 * ri;
                    A = fma(c23, ri3, ri);
                    B = ri3 * fma(-c2, ri2, 1.0);
                }
                const double dl = fma(dx, ls.x, fma(dy, ls.y, dz * ls.z));
                const double s = B * dl;
                ax[t] = fma(A, ls.x, fma(s, dx, ax[t]));
                ay[t] = fma(A, ls.y, fma(s, dy, ay[t]));
                az[t] = fma(A, ls.z, fma(s, dz, az[t]));
            }
        }
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int ti = it.t0 + threadIdx.x + t * 128;
        if (ti < ns) part[(long long)it.k * NBL + b0 + ti] = make_double4_32a(ax[t], ay[t], az[t], 0.0);
    }
}

void launch_rpy(gdc_ctx* c, int prec) {
    const int pe = prof_begin(c, prec == GDC_FP32_MIXED ? 0 : (prec == GDC_PREC_DF64 ? 3 : 1));
    if (prec == GDC_FP32_MIXED) {
        const double a = c->p.a;
        const RpyConst32 k = rpy_const32(a);
        // two targets per packed lane pair: tpt 4 -> P = 2, otherwise P = 1
#define GDC_RPY32_LAUNCH(PP, MB)                                                                             \
    k_rpy32<PP, MB><<<c->mv_n_items, 128, 0, c->stream>>>(c->mv_items, c->mv_active, c->susp_blob_off, c->spos, \
                                                          c->sdup, (float4*)c->mv_part, c->NBL, k, c->dev_status, \
                                                          first_wait_polls())
        if (c->use_sym) {
            launch_rpy32_sym(c);
        } else {
            ++c->n_launch;
            if (c->mv_tpt == 4) {
                if (c->mv_minb == 4)
                    GDC_RPY32_LAUNCH(2, 4);
                else
                    GDC_RPY32_LAUNCH(2, 6);
            } else {
                if (c->mv_minb == 4)
                    GDC_RPY32_LAUNCH(1, 4);
                else
                    GDC_RPY32_LAUNCH(1, 6);
            }
        }
#undef GDC_RPY32_LAUNCH
    } else if (prec == GDC_PREC_DF64 && c->dfs_minb) {
        launch_rpy_df_sym_pairs(c);   // its epilogue runs in launch_rpy_epilogue
    } else if (prec == GDC_PREC_DF64) {
        const RpyConstDF k = df_constants(c->p.a);
        if (c->mv_tpt == 4)
            ++c->n_launch, k_rpy_df<4><<<c->mv_n_items, 128, 0, c->stream>>>(c->mv_items, c->susp_blob_off, c->spos64,
                                                                             c->slam64, (double4_32a*)c->mv_part, c->NBL, k);
        else
            ++c->n_launch, k_rpy_df<2><<<c->mv_n_items, 128, 0, c->stream>>>(c->mv_items, c->susp_blob_off, c->spos64,
                                                                             c->slam64, (double4_32a*)c->mv_part, c->NBL, k);
    } else {
        if (c->mv_tpt == 1)
            ++c->n_launch, k_rpy64<1><<<c->mv_n_items, 128, 0, c->stream>>>(c->mv_items, c->mv_active, c->susp_blob_off, c->spos64, c->slam64,
                                                             (double4_32a*)c->mv_part, c->NBL, c->p.a);
        else if (c->mv_tpt == 4)
            ++c->n_launch, k_rpy64<4><<<c->mv_n_items, 128, 0, c->stream>>>(c->mv_items, c->mv_active, c->susp_blob_off, c->spos64, c->slam64,
                                                             (double4_32a*)c->mv_part, c->NBL, c->p.a);
        else
            ++c->n_launch, k_rpy64<2><<<c->mv_n_items, 128, 0, c->stream>>>(c->mv_items, c->mv_active, c->susp_blob_off, c->spos64, c->slam64,
                                                             (double4_32a*)c->mv_part, c->NBL, c->p.a);
    }
    prof_end(c, pe);
}

// ---- epilogue: chunk sums in FP64, scale, and the -K V part of the saddle operator ----

template <typename P>
__device__ inline void load_part(const P* part, long long idx, double& x, double& y, double& z) {
    const P v = part[idx];
    x = (double)v.x;
    y = (double)v.y;
    z = (double)v.z;
}

// Exact minus clamped pair coefficients (units of 1/(8 pi eta)) for a pair at distance r < 2a:
// the FP32 pair kernel evaluates every pair, the self pair and overlapping pairs included,
// with the far-field form at r clamped to 2a (A = 7/(12a), B = 1/(16a^3) there); the
// overlapping branch of the RPY tensor has A = 4/(3a) (1 - 9r/(32a)), B = 1/(8a^2 r).
// FP32 suffices: the correction joins a product whose pair terms are FP32.
__device__ inline void near_delta(float a, float r, float& dA, float& dB) {
    dA = 4.f / (3.f * a) * (1.f - 9.f * r / (32.f * a)) - 7.f / (12.f * a);
    dB = (r > 0.f ? 1.f / (8.f * a * a * r) : 0.f) - 1.f / (16.f * a * a * a);
}

// Adds to (ux, uy, uz), in units of 1/(8 pi eta), the exact minus clamped terms of blob i's
// pairs with blobs of other bodies closer than 2a: from the list when it holds them all, else
// by a search of the suspension's blobs [so, se) (FP64 distances; blob_body given: skip
// same-body blobs, else only j = i).  x holds lambda, 3 per blob, or in the saddle layout
// through gm (blob -> offset) when gm is given.
__device__ inline void near_pair_correction(long long i, long long so, long long se, const int* __restrict__ near_cnt,
                                            const int* __restrict__ near_idx, const int* __restrict__ blob_body,
                                            const double* __restrict__ r, const double* __restrict__ x,
                                            const int* __restrict__ gm, double a, double& ux, double& uy, double& uz) {
    const int m = near_cnt[i];
    const double four_a2 = 4.0 * a * a;
    const long long cnt = m <= GDC_NEAR_CAP ? m : se - so;
    for (long long q = 0; q < cnt; ++q) {
        const long long j = m <= GDC_NEAR_CAP ? (long long)near_idx[i * GDC_NEAR_CAP + q] : so + q;
        if (j == i || (blob_body && blob_body[j] == blob_body[i])) continue;
        const double dx = r[3 * j] - r[3 * i], dy = r[3 * j + 1] - r[3 * i + 1], dz = r[3 * j + 2] - r[3 * i + 2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < four_a2)) continue;   // at or beyond 2a the clamped form is the RPY tensor
        float dA, dB;
        near_delta((float)a, sqrtf((float)r2), dA, dB);
        const long long oj = gm ? (long long)gm[j] : 3LL * j;
        const double lx = x[oj], ly = x[oj + 1], lz = x[oj + 2];
        const double s = (double)dB * (dx * lx + dy * ly + dz * lz);
        ux += (double)dA * lx + s * dx;
        uy += (double)dA * ly + s * dy;
        uz += (double)dA * lz + s * dz;
    }
}

// Subtracts from (ux, uy, uz) the terms the FP32 pair kernel added for blob i's own body
// [j0, j1) (self pair included), recomputed from the same FP32 operands with the same
// operations, so that the FP32 rounding of those near-field terms cancels; the intra-body
// kernel then adds the same-body block of the body's template.
__device__ inline void same_body_subtract(const float4 pt, long long j0, long long j1, const float4* __restrict__ sdup,
                                          const RpyConst32& k, double& ux, double& uy, double& uz) {
    // summed in FP32 with compensation (FP64 adds are slow on GB300), subtracted once
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    auto kahan = [](float& sum, float& comp, float v) {
        const float y = __fsub_rn(v, comp);
        const float t = __fadd_rn(sum, y);
        comp = __fsub_rn(__fsub_rn(t, sum), y);
        sum = t;
    };
    for (long long j = j0; j < j1; ++j) {
        const float4 s0 = sdup[3 * j], s1 = sdup[3 * j + 1], s2 = sdup[3 * j + 2];
        const float dx = __fsub_rn(s0.x, pt.x), dy = __fsub_rn(s0.z, pt.y), dz = __fsub_rn(s1.x, pt.z);
        const float lx = s1.z, ly = s2.x, lz = s2.z;
        const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
        const float ri = rsqrtf(fmaxf(r2, k.four_a2));
        const float ri2 = __fmul_rn(ri, ri), ri3 = __fmul_rn(ri2, ri);
        const float A = __fmaf_rn(k.c23, ri3, ri);
        const float B = __fmul_rn(ri3, __fmaf_rn(-k.c2, ri2, 1.f));
        const float sj = __fmul_rn(B, __fmaf_rn(dx, lx, __fmaf_rn(dy, ly, __fmul_rn(dz, lz))));
        kahan(sx, cx, __fmaf_rn(A, lx, __fmul_rn(sj, dx)));
        kahan(sy, cy, __fmaf_rn(A, ly, __fmul_rn(sj, dy)));
        kahan(sz, cz, __fmaf_rn(A, lz, __fmul_rn(sj, dz)));
    }
    ux -= (double)sx - (double)cx;
    uy -= (double)sy - (double)cy;
    uz -= (double)sz - (double)cz;
}

// u_i = c0 (sum of the chunk partial sums [+ near-pair corrections]) [- K V]
//
// near_cnt != 0 (FP32 products): corrects the pairs of other bodies closer than 2a and takes
// out the pair kernel's same-body terms (the intra-body kernel adds the template's block).
template <typename P>
__global__ void k_rpy_epilogue(int NBL, const P* __restrict__ part, const int* __restrict__ blob_susp,
                               const int* __restrict__ nk, double c0, const double* __restrict__ x,
                               double* __restrict__ y, int gm_layout, const int* __restrict__ blob_gm,
                               const int* __restrict__ body_gm, const int* __restrict__ blob_body,
                               const double* __restrict__ r, const double* __restrict__ Yc,
                               const int* __restrict__ near_cnt, const int* __restrict__ near_idx, double a,
                               const long long* __restrict__ susp_blob_off, const long long* __restrict__ body_blob_off,
                               const float4* __restrict__ spos, const float4* __restrict__ sdup, RpyConst32 k32,
                               const float4* __restrict__ sym_part_j, const int* __restrict__ sym_row_nk,
                               const long long* __restrict__ sym_tile_base, const long long* __restrict__ sym_jbase) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    double ux = 0.0, uy = 0.0, uz = 0.0;
    if (sym_part_j) {
        // symmetric kernel: the target-side slots of the blob's tile row, then the source-side
        // slots (I, J) of every tile I before the blob's tile J, in order.  FP32 partials are
        // added with compensation in FP32 (GB300 adds in FP64 at a small fraction of the FP32
        // rate), then converted once.
        const int s = blob_susp[i];
        const long long loc = i - susp_blob_off[s];
        const int J = (int)(loc / GDC_SYM_TILE), e = (int)(loc % GDC_SYM_TILE);
        const int n = sym_row_nk[sym_tile_base[s] + J];
        const float4* pi = reinterpret_cast<const float4*>(part);
        float sx = 0.f, sy = 0.f, sz = 0.f, kx = 0.f, ky = 0.f, kz = 0.f;
        auto kahan = [](float& sum, float& comp, float v) {
            const float y = __fsub_rn(v, comp);
            const float t = __fadd_rn(sum, y);
            comp = __fsub_rn(__fsub_rn(t, sum), y);
            sum = t;
        };
        for (int k = 0; k < n; ++k) {
            const float4 v = pi[(long long)k * NBL + i];
            kahan(sx, kx, v.x);
            kahan(sy, ky, v.y);
            kahan(sz, kz, v.z);
        }
        const long long s0 = sym_jbase[s] + (long long)J * (J - 1) / 2;
        for (int I = 0; I < J; ++I) {
            const float4 v = sym_part_j[(s0 + I) * GDC_SYM_TILE + e];
            kahan(sx, kx, v.x);
            kahan(sy, ky, v.y);
            kahan(sz, kz, v.z);
        }
        ux = (double)sx - (double)kx;
        uy = (double)sy - (double)ky;
        uz = (double)sz - (double)kz;
    } else {
        const int n = nk[blob_susp[i]];
        for (int k = 0; k < n; ++k) {
            double a0, b, cc;
            load_part(part, (long long)k * NBL + i, a0, b, cc);
            ux += a0;
            uy += b;
            uz += cc;
        }
    }
    if (near_cnt) {
        const long long so = susp_blob_off[blob_susp[i]], se = susp_blob_off[blob_susp[i] + 1];
        near_pair_correction(i, so, se, near_cnt, near_idx, blob_body, r, x, gm_layout ? blob_gm : nullptr, a, ux, uy,
                             uz);
        const int p = blob_body[i];
        same_body_subtract(spos[i], body_blob_off[p], body_blob_off[p + 1], sdup, k32, ux, uy, uz);
    }
    ux *= c0;
    uy *= c0;
    uz *= c0;
    if (!gm_layout) {
        y[3 * i] = ux;
        y[3 * i + 1] = uy;
        y[3 * i + 2] = uz;
        return;
    }
    // saddle operator: M lambda - K V, K V = U_p + Omega_p x (r_i - Y_p)  (Eq. rigid_body_cond)
    const int p = blob_body[i];
    const double* V = x + body_gm[p];
    const double dx = r[3 * i] - Yc[3 * p], dy = r[3 * i + 1] - Yc[3 * p + 1], dz = r[3 * i + 2] - Yc[3 * p + 2];
    const double kx = V[0] + (V[4] * dz - V[5] * dy);
    const double ky = V[1] + (V[5] * dx - V[3] * dz);
    const double kz = V[2] + (V[3] * dy - V[4] * dx);
    const long long o = blob_gm[i];
    y[o] = ux - kx;
    y[o + 1] = uy - ky;
    y[o + 2] = uz - kz;
}

// Blob rows of the saddle operator with the FCM mobility: y_i = (M_FCM lambda)_i - (K V)_i,
// K V = U_p + Omega_p x (r_i - Y_p) (Eq. rigid_body_cond), u = M_FCM lambda given 3 per blob.
__global__ void k_fcm_saddle_rows(int NBL, const double* __restrict__ u, const double* __restrict__ x,
                                  double* __restrict__ y, const int* __restrict__ blob_gm, const int* __restrict__ body_gm,
                                  const int* __restrict__ blob_body, const double* __restrict__ r,
                                  const double* __restrict__ Yc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const int p = blob_body[i];
    const double* V = x + body_gm[p];
    const double dx = r[3 * i] - Yc[3 * p], dy = r[3 * i + 1] - Yc[3 * p + 1], dz = r[3 * i + 2] - Yc[3 * p + 2];
    const long long o = blob_gm[i];
    y[o] = u[3LL * i] - (V[0] + (V[4] * dz - V[5] * dy));
    y[o + 1] = u[3LL * i + 1] - (V[1] + (V[5] * dx - V[3] * dz));
    y[o + 2] = u[3LL * i + 2] - (V[2] + (V[3] * dy - V[4] * dx));
}

void launch_fcm_saddle_rows(gdc_ctx* c, const double* x, double* y) {
    ++c->n_launch, k_fcm_saddle_rows<<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(
        c->NBL, c->fcm_u, x, y, c->blob_gm, c->body_gm, c->blob_body, c->r, c->Yc);
}

static void launch_epilogue(gdc_ctx* c, int prec, double c0, const double* x, double* y, int gm_layout,
                            bool near) {
    const bool sym = prec == GDC_FP32_MIXED && near && c->use_sym;   // RPY products only, not forces
    if (prec == GDC_FP32_MIXED)
        ++c->n_launch, k_rpy_epilogue<float4><<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(
            c->NBL, sym ? c->sym_part_i : (const float4*)c->mv_part, c->blob_susp, c->mv_nk, c0, x, y, gm_layout,
            c->blob_gm, c->body_gm, c->blob_body, c->r, c->Yc, near ? c->near_cnt : nullptr, c->near_idx, c->p.a,
            c->susp_blob_off, c->body_blob_off, c->spos, c->sdup, rpy_const32(c->p.a), sym ? c->sym_part_j : nullptr,
            c->sym_row_nk, c->sym_tile_base, c->sym_jbase);
    else
        ++c->n_launch, k_rpy_epilogue<double4_32a><<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(
            c->NBL, (const double4_32a*)c->mv_part, c->blob_susp, c->mv_nk, c0, x, y, gm_layout, c->blob_gm, c->body_gm,
            c->blob_body, c->r, c->Yc, nullptr, nullptr, c->p.a, c->susp_blob_off, c->body_blob_off, c->spos, c->sdup,
            rpy_const32(c->p.a), nullptr, nullptr, nullptr, nullptr);
}

void launch_rpy_epilogue(gdc_ctx* c, int prec, const double* x, double* y, int gm_layout, bool same_body) {
    if (prec == GDC_PREC_DF64 && c->dfs_minb)
        launch_rpy_df_sym_epilogue(c, x, y, gm_layout);
    else
        launch_epilogue(c, prec, 1.0 / (8.0 * 3.141592653589793 * c->p.eta), x, y, gm_layout, prec == GDC_FP32_MIXED);
    // same-body blocks from the template: the df64 pair kernel leaves those pairs out and the
    // FP32 epilogue has taken the FP32 pair kernel's same-body terms out again (so without
    // them an FP32 product is exactly the blocks between different bodies)
    if (prec == GDC_PREC_DF64) launch_intra_body(c, x, y, gm_layout);
    if (prec == GDC_FP32_MIXED && same_body) launch_intra_body32(c, x, y, gm_layout);
}

// ---- pairs closer than 2a ------------------------------------------------------------

// For every blob i, the blobs j of other bodies of its suspension whose FP32 r_ij^2, computed
// exactly as the FP32 pair kernel computes it, is below 4a^2 -- the pairs the pair kernel
// clamps: the pairs whose term the epilogue corrects (same-body pairs are replaced whole).  One block per (256 targets, source chunk) of one
// suspension, two targets per thread in packed arithmetic; a found pair takes the next slot
// of its target's list (near_cnt starts at zero), and k_near_sort then orders every list so
// that the corrections are summed in a fixed order.
__global__ void __launch_bounds__(128) k_near_build(const int4* __restrict__ items, const long long* __restrict__ susp_blob_off,
                                                   const float4* __restrict__ spos, float four_a2,
                                                   int* __restrict__ near_cnt, int* __restrict__ near_idx) {
    __shared__ float4 sh[2 * 256];
    const int4 it = items[blockIdx.x];   // (suspension, first target, first source, end source)
    const long long b0 = susp_blob_off[it.x];
    const int ns = (int)(susp_blob_off[it.x + 1] - b0);
    const int ta = it.y + (int)threadIdx.x, tb = ta + 128;
    const float4 pa = spos[b0 + min(ta, ns - 1)], pb = spos[b0 + min(tb, ns - 1)];
    const float2 xt = make_float2(pa.x, pb.x), yt = make_float2(pa.y, pb.y), zt = make_float2(pa.z, pb.z);
    for (int j0 = it.z; j0 < it.w; j0 += 256) {
        const int n = min(256, it.w - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < n; e += 128) {
            const float4 q = spos[b0 + j0 + e];
            sh[2 * e] = make_float4(q.x, q.x, q.y, q.y);
            sh[2 * e + 1] = make_float4(q.z, q.z, q.w, q.w);   // w: body index bits
        }
        __syncthreads();
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            const float4 s0 = sh[2 * j], s1 = sh[2 * j + 1];
            const float2 dx = sub2(make_float2(s0.x, s0.y), xt), dy = sub2(make_float2(s0.z, s0.w), yt),
                         dz = sub2(make_float2(s1.x, s1.y), zt);
            const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
            if (r2.x < four_a2 || r2.y < four_a2) {   // rare
                const int jg = j0 + j;
                const int bj = __float_as_int(s1.z);
                if (r2.x < four_a2 && bj != __float_as_int(pa.w) && ta < ns) {
                    const int slot = atomicAdd(near_cnt + b0 + ta, 1);
                    if (slot < GDC_NEAR_CAP) near_idx[(b0 + ta) * GDC_NEAR_CAP + slot] = (int)(b0 + jg);
                }
                if (r2.y < four_a2 && bj != __float_as_int(pb.w) && tb < ns) {
                    const int slot = atomicAdd(near_cnt + b0 + tb, 1);
                    if (slot < GDC_NEAR_CAP) near_idx[(b0 + tb) * GDC_NEAR_CAP + slot] = (int)(b0 + jg);
                }
            }
        }
    }
}

// Orders each blob's near-pair list (insertion sort; lists are short).  A count above
// GDC_NEAR_CAP leaves the list incomplete: the epilogue then searches the suspension.
__global__ void k_near_sort(int n, const int* __restrict__ near_cnt, int* __restrict__ near_idx) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int m = near_cnt[i];
    if (m < 2 || m > GDC_NEAR_CAP) return;
    int* l = near_idx + i * GDC_NEAR_CAP;
    for (int a = 1; a < m; ++a) {
        const int v = l[a];
        int b = a - 1;
        while (b >= 0 && l[b] > v) {
            l[b + 1] = l[b];
            --b;
        }
        l[b + 1] = v;
    }
}

void launch_near_build(gdc_ctx* c) {
    if (c->p.mobility == GDC_MOB_FCM) return;   // the lists serve the RPY products only
    if (forces_use_cells(c)) {
        launch_near_cell(c);   // the same lists from a cell list, O(N_b)
    } else {
        cudaMemsetAsync(c->near_cnt, 0, sizeof(int) * c->NBL, c->stream);
        ++c->n_launch, k_near_build<<<c->n_near_items, 128, 0, c->stream>>>(c->near_items, c->susp_blob_off, c->spos,
                                                                            (float)(4.0 * c->p.a * c->p.a), c->near_cnt,
                                                                            c->near_idx);
    }
    ++c->n_launch, k_near_sort<<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(c->NBL, c->near_cnt, c->near_idx);
}

// ---- pair forces between blobs of different bodies, every pair in tiles -------------

// f_i = sum_j F(|r_i - r_j|) (r_i - r_j)/|r_i - r_j| over blobs j of other bodies with F
// the pair force of forces.cuh; pairs beyond its cutoff are skipped.
template <int TPT>
__global__ void __launch_bounds__(128) k_forces32(const MvItem* __restrict__ items, const long long* __restrict__ susp_blob_off,
                                                  const float4* __restrict__ spos, float4* __restrict__ part, int NBL,
                                                  ForceK<float> k) {
    __shared__ float4 sp[MV_TILE];
    const MvItem it = items[blockIdx.x];
    const long long b0 = susp_blob_off[it.s];
    const int ns = (int)(susp_blob_off[it.s + 1] - b0);
    const int ti0 = it.t0 + threadIdx.x;
    float xt[TPT], yt[TPT], zt[TPT], fx[TPT], fy[TPT], fz[TPT];
    int bt[TPT];
    for (int t = 0; t < TPT; ++t) {
        fx[t] = fy[t] = fz[t] = 0.f;
        const float4 p = spos[b0 + min(ti0 + t * 128, ns - 1)];
        xt[t] = p.x;
        yt[t] = p.y;
        zt[t] = p.z;
        bt[t] = __float_as_int(p.w);
    }
    for (int j0 = it.j0; j0 < it.j1; j0 += MV_TILE) {
        const int n = min(MV_TILE, it.j1 - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < n; e += 128) sp[e] = spos[b0 + j0 + e];
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const float4 ps = sp[j];
            const int bj = __float_as_int(ps.w);
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                const float dx = xt[t] - ps.x, dy = yt[t] - ps.y, dz = zt[t] - ps.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (bj != bt[t] && r2 < k.rc2 && r2 > 0.f) {
                    const float r = sqrtf(r2);
                    const float s = pair_force(r, k) / r;
                    fx[t] = fmaf(s, dx, fx[t]);
                    fy[t] = fmaf(s, dy, fy[t]);
                    fz[t] = fmaf(s, dz, fz[t]);
                }
            }
        }
    }
    for (int t = 0; t < TPT; ++t) {
        const int ti = ti0 + t * 128;
        if (ti < ns) part[(long long)it.k * NBL + b0 + ti] = make_float4(fx[t], fy[t], fz[t], 0.f);
    }
}

template <int TPT>
__global__ void __launch_bounds__(128) k_forces64(const MvItem* __restrict__ items, const long long* __restrict__ susp_blob_off,
                                                  const double4_32a* __restrict__ spos, double4_32a* __restrict__ part, int NBL,
                                                  ForceK<double> k) {
    __shared__ double4_32a sp[MV_TILE];
    const MvItem it = items[blockIdx.x];
    const long long b0 = susp_blob_off[it.s];
    const int ns = (int)(susp_blob_off[it.s + 1] - b0);
    const int ti0 = it.t0 + threadIdx.x;
    double xt[TPT], yt[TPT], zt[TPT], fx[TPT], fy[TPT], fz[TPT];
    long long bt[TPT];
    for (int t = 0; t < TPT; ++t) {
        fx[t] = fy[t] = fz[t] = 0.0;
        const double4_32a p = spos[b0 + min(ti0 + t * 128, ns - 1)];
        xt[t] = p.x;
        yt[t] = p.y;
        zt[t] = p.z;
        bt[t] = (long long)p.w;
    }
    for (int j0 = it.j0; j0 < it.j1; j0 += MV_TILE) {
        const int n = min(MV_TILE, it.j1 - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < n; e += 128) sp[e] = spos[b0 + j0 + e];
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const double4_32a ps = sp[j];
            const long long bj = (long long)ps.w;
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                const double dx = xt[t] - ps.x, dy = yt[t] - ps.y, dz = zt[t] - ps.z;
                const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                if (bj != bt[t] && r2 < k.rc2 && r2 > 0.0) {
                    const double r = sqrt(r2);
                    const double s = pair_force(r, k) / r;
                    fx[t] = fma(s, dx, fx[t]);
                    fy[t] = fma(s, dy, fy[t]);
                    fz[t] = fma(s, dz, fz[t]);
                }
            }
        }
    }
    for (int t = 0; t < TPT; ++t) {
        const int ti = ti0 + t * 128;
        if (ti < ns) part[(long long)it.k * NBL + b0 + ti] = make_double4_32a(fx[t], fy[t], fz[t], 0.0);
    }
}

#define GDC_FORCES_LAUNCH(TPT)                                                                         \
    do {                                                                                               \
        if (prec == GDC_FP32_MIXED)                                                                    \
            ++c->n_launch, k_forces32<TPT><<<c->mv_n_items, 128, 0, c->stream>>>(c->mv_items, c->susp_blob_off, c->spos, \
                (float4*)c->mv_part, c->NBL, force_constants<float>(c->p));                                \
        else                                                                                           \
            ++c->n_launch, k_forces64<TPT><<<c->mv_n_items, 128, 0, c->stream>>>(c->mv_items, c->susp_blob_off,          \
                c->spos64, (double4_32a*)c->mv_part, c->NBL, force_constants<double>(c->p));                   \
    } while (0)

void launch_forces_pair(gdc_ctx* c, int prec, double* fblob) {
    const int pe = prof_begin(c, 2);
    if (c->mv_tpt == 1)
        GDC_FORCES_LAUNCH(1);
    else if (c->mv_tpt == 4)
        GDC_FORCES_LAUNCH(4);
    else
        GDC_FORCES_LAUNCH(2);
    prof_end(c, pe);
    launch_epilogue(c, prec, 1.0, nullptr, fblob, 0, false);
}

// ---- work list ------------------------------------------------------------------------

void build_mv_items(gdc_ctx* c, int tpt, double waves) {
    c->mv_tpt = tpt;
    c->mv_waves = waves;
    const int tile_targets = 128 * tpt;
    double P = 0.0;
    std::vector<long long> ns(c->S);
    for (int s = 0; s < c->S; ++s) {
        ns[s] = c->h_blob_off[s + 1] - c->h_blob_off[s];
        P += (double)ns[s] * (double)ns[s];
    }
    c->pair_evals_per_matvec = P;
    const double target_items = (double)c->num_sms * 4.0 * waves;  // `waves` launches of 4 blocks per SM
    c->h_mv_items.clear();
    c->h_mv_nk.assign(c->S, 1);
    int kmax = 1;
    for (int s = 0; s < c->S; ++s) {
        const long long n = ns[s];
        const int nt = ceil_div(n, tile_targets);
        int nk = (int)std::lround(target_items * (double)n * (double)n / std::max(P, 1.0) / std::max(nt, 1));
        nk = std::max(1, std::min(nk, std::max(1, ceil_div(n, 512))));
        nk = std::min(nk, 64);
        long long csz = (n + nk - 1) / nk;
        csz = ((csz + 31) / 32) * 32;
        nk = (int)std::max<long long>(1, (n + csz - 1) / csz);
        c->h_mv_nk[s] = nk;
        kmax = std::max(kmax, nk);
        for (int t = 0; t < nt; ++t)
            for (int k = 0; k < nk; ++k) {
                MvItem it{};
                it.s = s;
                it.t0 = t * tile_targets;
                it.j0 = (int)(k * csz);
                it.j1 = (int)std::min<long long>(n, (k + 1) * csz);
                it.k = k;
                if (it.j1 > it.j0) c->h_mv_items.push_back(it);
            }
    }
    // largest items first, so the tail of the launch is made of small ones
    std::stable_sort(c->h_mv_items.begin(), c->h_mv_items.end(), [&](const MvItem& x, const MvItem& y) {
        const long long cx = (long long)std::min<long long>(tile_targets, ns[x.s] - x.t0) * (x.j1 - x.j0);
        const long long cy = (long long)std::min<long long>(tile_targets, ns[y.s] - y.t0) * (y.j1 - y.j0);
        return cx > cy;
    });
    c->mv_n_items = (int)c->h_mv_items.size();
    c->mv_kmax = kmax;
}

}  // namespace gdc

namespace gdc {

// Candidate tilings of the pair kernels: targets per thread x work items per launch.
static const int kTpt[2] = {2, 4};
static const double kWaves[3] = {4.0, 8.0, 16.0};
static const int kSymWidth[3] = {2, 4, 8};   // source tiles per item of the symmetric kernel
static const int kSymMinBlocks[3] = {2, 3, 4};   // resident blocks per SM of the symmetric kernel
static const int kMvMinBlocks[2] = {4, 6};       // resident blocks per SM of the ordered kernel
static const int kDfsMinBlocks[3] = {0, 3, 4};   // double-float kernel: ordered, symmetric at 3 or 4 per SM

void plan_mv_capacity(gdc_ctx* c) {
    int cap_items = 0, cap_k = 1;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            build_mv_items(c, kTpt[a], kWaves[b]);
            cap_items = std::max(cap_items, c->mv_n_items);
            cap_k = std::max(cap_k, c->mv_kmax);
        }
    c->mv_cap_items = cap_items;
    c->mv_cap_kmax = cap_k;
    build_mv_items(c, 2, 8.0);
    int scap = 0, sk = 1;
    for (int w : kSymWidth) {
        build_sym_items(c, w);
        scap = std::max(scap, c->sym_n_items);
        sk = std::max(sk, c->sym_kmax);
    }
    c->sym_cap_items = scap;
    c->sym_cap_kmax = sk;
    c->sym_n_tiles = c->h_sym_tile_base.back();
    c->sym_n_jslots = c->h_sym_jbase.back();
    build_sym_items(c, 4);
    // the symmetric double-float kernel: items of GDC_DFS_WIDTH source tiles, so that with 3
    // or 4 resident blocks per SM the last wave of long items stays full; wider in
    // suspensions of more than 64 x GDC_DFS_WIDTH tiles, which keeps the target-side slots
    // at 64 per blob (each wave is then a small part of the launch anyway)
    int tmax = 1;
    for (int s = 0; s < c->S; ++s)
        tmax = std::max(tmax, (int)((c->h_blob_off[s + 1] - c->h_blob_off[s] + GDC_SYM_TILE - 1) / GDC_SYM_TILE));
    build_sym_list(c, std::max(GDC_DFS_WIDTH, (tmax + 63) / 64), c->h_dfs_items, c->h_dfs_row_nk, c->dfs_kmax);
    c->dfs_n_items = (int)c->h_dfs_items.size();
}

static gdc_status upload_items(gdc_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->mv_items, c->h_mv_items.data(), sizeof(MvItem) * c->h_mv_items.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->mv_nk, c->h_mv_nk.data(), sizeof(int) * c->S, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "work-list upload");
}

// Times three launches of the FP32 RPY kernel per candidate at the loaded configuration
// (lambda = the current W buffer) and keeps the fastest tiling; then one launch of each
// double-float residual kernel.
gdc_status autotune_pair_kernel(gdc_ctx* c) {
    cudaEvent_t e0, e1;
    gdc_status st = cuda_check(c, cudaEventCreate(&e0), "event");
    if (st != GDC_OK) return st;
    if ((st = cuda_check(c, cudaEventCreate(&e1), "event")) != GDC_OK) return st;
    launch_normals(c, 0, 0, c->W);
    launch_pack_lambda(c, GDC_FP32_MIXED, c->W, 0);
    const int only = c->p.pair_kernel;   // 0: both kernels, 1: ordered, 2: symmetric
    float best = 1e30f;
    int bt = 2, bsym = 0, bwid = 4;
    double bw = 8.0;
    auto time3 = [&](float& ms) -> gdc_status {
        launch_rpy(c, GDC_FP32_MIXED);  // warm-up
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3; ++r) launch_rpy(c, GDC_FP32_MIXED);
        cudaEventRecord(e1, c->stream);
        gdc_status s2 = cuda_check(c, cudaEventSynchronize(e1), "autotune");
        if (s2 == GDC_OK) cudaEventElapsedTime(&ms, e0, e1);
        return s2;
    };
    int bmv_minb = 6;
    if (only != 2) {
        c->use_sym = 0;
        for (int a = 0; a < 2 && st == GDC_OK; ++a)
            for (int b = 0; b < 3 && st == GDC_OK; ++b) {
                build_mv_items(c, kTpt[a], kWaves[b]);
                if ((st = upload_items(c)) != GDC_OK) break;
                for (int mb : kMvMinBlocks) {
                    c->mv_minb = mb;
                    float ms = 0.f;
                    if ((st = time3(ms)) != GDC_OK) break;
                    if (ms < best) {
                        best = ms;
                        bt = kTpt[a];
                        bw = kWaves[b];
                        bmv_minb = mb;
                        bsym = 0;
                    }
                }
            }
    }
    int bminb = 2;
    if (only != 1 && st == GDC_OK) {
        c->use_sym = 1;
        for (int w : kSymWidth) {
            build_sym_items(c, w);
            if ((st = sym_upload(c)) != GDC_OK) break;
            for (int mb : kSymMinBlocks) {
                c->sym_minb = mb;
                float ms = 0.f;
                if ((st = time3(ms)) != GDC_OK) break;
                if (ms < best) {
                    best = ms;
                    bwid = w;
                    bminb = mb;
                    bsym = 1;
                }
            }
            if (st != GDC_OK) break;
        }
    }
    if (st == GDC_OK) {
        build_mv_items(c, bt, bw);
        build_sym_items(c, bwid);
        c->use_sym = bsym;
        c->sym_minb = bminb;
        c->mv_minb = bmv_minb;
        c->autotune_ms = best / 3.0;
        st = upload_items(c);
        if (st == GDC_OK) st = sym_upload(c);
    }
    // the double-float residual kernel, one timed launch each after a warm-up (about 40 ms
    // per product at 65k blobs): ordered unless the FP32 kernel is pinned to symmetric
    c->dfs_minb = only == 1 ? 0 : 4;
    if (c->p.df_kernel) {
        c->dfs_minb = c->p.df_kernel == 1 ? 0 : c->p.df_kernel;
    } else if (only != 1 && st == GDC_OK) {
        launch_pack_lambda(c, GDC_PREC_DF64, c->W, 0);
        float dbest = 1e30f;
        int bdf = 4;
        for (int mb : kDfsMinBlocks) {
            if (mb == 0 && only == 2) continue;
            c->dfs_minb = mb;
            float ms = 0.f;
            launch_rpy(c, GDC_PREC_DF64);   // warm-up
            cudaEventRecord(e0, c->stream);
            launch_rpy(c, GDC_PREC_DF64);
            cudaEventRecord(e1, c->stream);
            if ((st = cuda_check(c, cudaEventSynchronize(e1), "autotune")) != GDC_OK) break;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < dbest) {
                dbest = ms;
                bdf = mb;
            }
        }
        c->dfs_minb = bdf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// Without the autotuner: the kernel params.pair_kernel names (symmetric for 0 and 2) with
// the default work lists, and the double-float kernel of the same kind.
gdc_status default_pair_kernel(gdc_ctx* c) {
    c->use_sym = c->p.pair_kernel != 1;
    c->dfs_minb = c->p.df_kernel ? (c->p.df_kernel == 1 ? 0 : c->p.df_kernel) : (c->use_sym ? 4 : 0);
    gdc_status st = upload_items(c);
    return st != GDC_OK ? st : sym_upload(c);
}

}  // namespace gdc

// ---- allocation-free RPY product (gdc_rpy_apply_noalloc) ------------------------------
//
// For callers that cannot allocate device memory.  All scratch of this variant (packed
// sources, chunk partial sums, the work list) lives in one file-scope device array of
// fixed size, so the call allocates nothing; every GPU that loads the library holds the
// array until the process exits.  It reuses the FP32 pair kernel above on one suspension
// of free blobs, with the same near-pair list and FP64 corrections of the self pair and of
// the pairs closer than 2a.

#include <mutex>

#define GDC_NOALLOC_MAX_CHUNKS 16
#define GDC_NOALLOC_TILE 256   // targets per work item (two per thread)

namespace gdc {

struct NoallocScratch {
    float4 spos[GDC_NOALLOC_MAX_BLOBS];
    float4 sdup[3 * GDC_NOALLOC_MAX_BLOBS];
    float4 part[GDC_NOALLOC_MAX_CHUNKS * GDC_NOALLOC_MAX_BLOBS];
    MvItem items[(GDC_NOALLOC_MAX_BLOBS / GDC_NOALLOC_TILE) * GDC_NOALLOC_MAX_CHUNKS];
    int4 near_items[(GDC_NOALLOC_MAX_BLOBS / 256) * (GDC_NOALLOC_MAX_BLOBS / GDC_NEAR_SRC)];
    int near_cnt[GDC_NOALLOC_MAX_BLOBS];
    int near_idx[GDC_NOALLOC_MAX_BLOBS * GDC_NEAR_CAP];
    long long susp_blob_off[2];
    double cen[3];   // blob centroid of the call (the FP32 positions are taken relative to it)
    int status[4];   // set by the pair kernel if a tile copy times out (u is then incomplete)
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Start of a call: the blob centroid (one block; per-thread strided sums added in a fixed
// tree order, so the result does not depend on timing) and the status words cleared.
__global__ void __launch_bounds__(256) k_noalloc_begin(NoallocScratch* __restrict__ sc, const double* __restrict__ r,
                                                       int n) {
    __shared__ double part[3][256];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += 256)
        for (int d = 0; d < 3; ++d) acc[d] += r[3 * i + d];
    for (int d = 0; d < 3; ++d) part[d][threadIdx.x] = acc[d];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int d = 0; d < 3; ++d) part[d][threadIdx.x] += part[d][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) sc->cen[threadIdx.x] = part[threadIdx.x][0] / n;
    if (threadIdx.x < 4) sc->status[threadIdx.x] = 0;
}

// Positions relative to the blob centroid (FP32), lambda, identity body table, work list.
__global__ void k_noalloc_prepare(NoallocScratch* __restrict__ sc, const double* __restrict__ r,
                                  const double* __restrict__ lam, int n, int nk, int csz) {
    const double c0 = sc->cen[0], c1 = sc->cen[1], c2 = sc->cen[2];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        sc->near_cnt[i] = 0;
        if (i % 256 == 0)   // near-pair blocks: 256 targets x source chunks of GDC_NEAR_SRC
            for (int j0 = 0, q = 0; j0 < n; j0 += GDC_NEAR_SRC, ++q)
                sc->near_items[(i / 256) * ((n + GDC_NEAR_SRC - 1) / GDC_NEAR_SRC) + q] =
                    make_int4(0, i, j0, min(n, j0 + GDC_NEAR_SRC));
        const float x = (float)(r[3 * i] - c0), y = (float)(r[3 * i + 1] - c1), z = (float)(r[3 * i + 2] - c2);
        const float lx = (float)lam[3 * i], ly = (float)lam[3 * i + 1], lz = (float)lam[3 * i + 2];
        sc->spos[i] = make_float4(x, y, z, __int_as_float(i));
        sc->sdup[3 * i] = make_float4(x, x, y, y);
        sc->sdup[3 * i + 1] = make_float4(z, z, lx, lx);
        sc->sdup[3 * i + 2] = make_float4(ly, ly, lz, lz);
    }
    const int ntile = (n + GDC_NOALLOC_TILE - 1) / GDC_NOALLOC_TILE;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < ntile * nk; b += gridDim.x * blockDim.x) {
        MvItem it{};
        it.s = 0;
        it.t0 = (b / nk) * GDC_NOALLOC_TILE;
        it.k = b % nk;
        it.j0 = it.k * csz;
        it.j1 = min(n, (it.k + 1) * csz);
        sc->items[b] = it;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->susp_blob_off[0] = 0;
        sc->susp_blob_off[1] = n;
    }
}

// u_i = c0 (sum of chunk partials + self-pair and near-pair corrections)
__global__ void k_noalloc_epilogue(const NoallocScratch* __restrict__ sc, const double* __restrict__ r,
                                   const double* __restrict__ lam, int n, int nk, double c0, double a,
                                   double* __restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (sc->status[1] != 0) {   // a tile copy of the pair kernel timed out: u would be incomplete
        u[3 * i] = u[3 * i + 1] = u[3 * i + 2] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    double x = 0.0, y = 0.0, z = 0.0;
    for (int k = 0; k < nk; ++k) {
        const float4 v = sc->part[(long long)k * GDC_NOALLOC_MAX_BLOBS + i];
        x += v.x;
        y += v.y;
        z += v.z;
    }
    // self pair: exact 4/(3a), clamped far field 7/(12a) (d = 0, so FP32 leaves only the rsqrt rounding)
    const double cs = 4.0 / (3.0 * a) - 7.0 / (12.0 * a);
    x += cs * lam[3 * i];
    y += cs * lam[3 * i + 1];
    z += cs * lam[3 * i + 2];
    near_pair_correction(i, 0, n, sc->near_cnt, sc->near_idx, nullptr, r, lam, nullptr, a, x, y, z);
    u[3 * i] = c0 * x;
    u[3 * i + 1] = c0 * y;
    u[3 * i + 2] = c0 * z;
}

// Device address of the scratch array and SM count, looked up once per device.
static std::mutex g_noalloc_mu;
static NoallocScratch* g_noalloc_ptr[128] = {};
static int g_noalloc_sms[128] = {};
static thread_local std::string g_noalloc_err;

const char* noalloc_last_error() { return g_noalloc_err.c_str(); }

static gdc_status noalloc_fail(gdc_status s, const std::string& m) {
    g_noalloc_err = m;
    return s;
}

}  // namespace gdc

extern "C" gdc_status gdc_rpy_apply_noalloc(const double* r, const double* lambda, double* u, int n_blobs, double a,
                                            double eta, void* stream) {
    using namespace gdc;
    if (!r || !lambda || !u) return noalloc_fail(GDC_ERR_INVALID_ARG, "gdc_rpy_apply_noalloc: NULL pointer");
    if (n_blobs < 1 || n_blobs > GDC_NOALLOC_MAX_BLOBS)
        return noalloc_fail(GDC_ERR_INVALID_ARG, "gdc_rpy_apply_noalloc: n_blobs must be in [1, " +
                                                     std::to_string(GDC_NOALLOC_MAX_BLOBS) + "], got " +
                                                     std::to_string(n_blobs));
    if (!(a > 0.0) || !(eta > 0.0)) return noalloc_fail(GDC_ERR_INVALID_ARG, "gdc_rpy_apply_noalloc: a and eta must be > 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128)
        return noalloc_fail(GDC_ERR_CUDA, std::string("gdc_rpy_apply_noalloc: no usable device: ") + cudaGetErrorString(e));
    NoallocScratch* sc;
    int sms;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {   // first call on this device: look up the array's device address
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(GDC_ERR_CUDA, std::string("gdc_rpy_apply_noalloc: cudaGetSymbolAddress failed: ") +
                                                      cudaGetErrorString(e));
            int v = 0;
            if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
            g_noalloc_sms[dev] = v;
            g_noalloc_ptr[dev] = (NoallocScratch*)p;
        }
        sc = g_noalloc_ptr[dev];
        sms = g_noalloc_sms[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int ntile = (n_blobs + GDC_NOALLOC_TILE - 1) / GDC_NOALLOC_TILE;
    int nk = std::max(1, std::min(GDC_NOALLOC_MAX_CHUNKS, (8 * sms + ntile - 1) / ntile));
    nk = std::min(nk, std::max(1, (n_blobs + 255) / 256));
    int csz = (n_blobs + nk - 1) / nk;
    csz = (csz + 31) / 32 * 32;
    nk = (n_blobs + csz - 1) / csz;
    k_noalloc_begin<<<1, 256, 0, st>>>(sc, r, n_blobs);
    k_noalloc_prepare<<<std::min(1024, (n_blobs + 255) / 256 + 1), 256, 0, st>>>(sc, r, lambda, n_blobs, nk, csz);
    RpyConst32 k{(float)(2.0 * a * a / 3.0), (float)(2.0 * a * a), (float)(4.0 * a * a), (float)(4.0 / (3.0 * a)),
                 (float)(9.0 / (32.0 * a)), (float)(1.0 / (8.0 * a * a))};
    // the pair kernel addresses partial sums as part[k * NBL + i]: pass the array's row length
    const int near_chunks = (n_blobs + GDC_NEAR_SRC - 1) / GDC_NEAR_SRC;
    k_near_build<<<((n_blobs + 255) / 256) * near_chunks, 128, 0, st>>>(sc->near_items, sc->susp_blob_off, sc->spos,
                                                                       (float)(4.0 * a * a), sc->near_cnt, sc->near_idx);
    k_near_sort<<<(n_blobs + 255) / 256, 256, 0, st>>>(n_blobs, sc->near_cnt, sc->near_idx);
    k_rpy32<1, 6><<<ntile * nk, 128, 0, st>>>(sc->items, nullptr, sc->susp_blob_off, sc->spos, sc->sdup, sc->part,
                                             GDC_NOALLOC_MAX_BLOBS, k, sc->status, first_wait_polls());
    k_noalloc_epilogue<<<(n_blobs + 255) / 256, 256, 0, st>>>(sc, r, lambda, n_blobs, nk,
                                                              1.0 / (8.0 * 3.141592653589793 * eta), a, u);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return noalloc_fail(GDC_ERR_CUDA, std::string("gdc_rpy_apply_noalloc: launch failed: ") + cudaGetErrorString(e));
    return GDC_OK;
}
