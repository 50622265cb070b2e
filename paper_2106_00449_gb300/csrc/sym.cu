// Symmetric FP32 RPY pair kernel: every unordered pair of blobs is evaluated once and
// contributes to both blobs (the RPY tensor is symmetric, M_ij = M_ji, and even in
// d = r_j - r_i), which removes a quarter of the FMA-pipe work of the ordered kernel: per
// unordered pair the distance and the coefficients A, B are shared and only the two
// products with lambda_j and lambda_i remain.
//
// A suspension's blobs are cut into tiles of SYM_TILE.  A block takes target tile I against
// source tiles J0..J1-1 (J >= I).  The diagonal tile J = I is evaluated ordered (every
// ordered pair, i-side only).  For J > I each warp holds 128 targets (four per lane, two
// packed pairs); a 32-source sub-chunk is swept in 32 steps in which lane l reads source
// (l + step) mod 32 from shared memory, so that the 32 lanes hold 32 different sources, and
// the source-side sum travels with its source: after every step the lanes pass their
// source accumulators one lane down with a shuffle, and after 32 steps each accumulator is
// back at the lane of its source.  The four warps' source-side sums of a tile are added in
// warp order and written to one slot per (I, J): the sums are deterministic.
//
// Pairs are evaluated exactly as the ordered kernel evaluates them (clamped distance
// max(r, 2a), same operations), so the epilogue's near-pair and same-body corrections
// apply unchanged.
#include <algorithm>

#include "common.cuh"
#include "pair_common.cuh"

namespace gdc {

constexpr int SYM_TILE = GDC_SYM_TILE;
constexpr int SYM_SMEM = 3 * SYM_TILE * 16 + 3 * 4 * SYM_TILE * 4 + 16;   // tile, 4 warps' sums, mbarrier

// Resident blocks per SM the register allocator is asked to allow (MINB): 2 (184 registers),
// 3 (165) or 4 (126), none spilling; the autotuner times each with each work-item width.

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_rpy32_sym(const SymItem* __restrict__ items,
                                                                 const int* __restrict__ active,
                                                                 const long long* __restrict__ susp_blob_off,
                                                                 const long long* __restrict__ jbase,
                                                                 const float4* __restrict__ spos,
                                                                 const float4* __restrict__ sdup,
                                                                 float4* __restrict__ part_i, float4* __restrict__ part_j,
                                                                 int NBL, RpyConst32 k, int* __restrict__ status,
                                                                 int first_polls) {
    extern __shared__ __align__(128) float4 dsm[];
    float4* sh = dsm;                                             // the source tile, sdup layout
    float* jsx = reinterpret_cast<float*>(dsm + 3 * SYM_TILE);    // [warp][source] source-side sums
    float* jsy = jsx + 4 * SYM_TILE;
    float* jsz = jsy + 4 * SYM_TILE;
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(jsz + 4 * SYM_TILE);
    const SymItem it = items[blockIdx.x];
    const long long b0 = susp_blob_off[it.s];
    const int ns = (int)(susp_blob_off[it.s + 1] - b0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tbase = it.I * SYM_TILE;
    if (active && !active[it.s]) {
        // a suspension whose Krylov loop has stopped: its product is not used; leave zeros
        for (int t = threadIdx.x; t < SYM_TILE && tbase + t < ns; t += 128)
            part_i[(long long)it.k * NBL + b0 + tbase + t] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int J = max(it.J0, it.I + 1); J < it.J1; ++J) {
            const long long slot = jbase[it.s] + (long long)J * (J - 1) / 2 + it.I;
            for (int e = threadIdx.x; e < SYM_TILE; e += 128)
                part_j[slot * SYM_TILE + e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    const float2 c23 = make_float2(k.c23, k.c23), mc2 = make_float2(-k.c2, -k.c2), one = make_float2(1.f, 1.f);
    const float four_a2 = k.four_a2;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // targets tbase + threadIdx.x + 128 m, m = 0..3; packed pair p holds m = 2p (x) and 2p + 1 (y).
    // A target past the end of the suspension sits on the last blob with lambda = 0, so it
    // adds nothing to any source; its own sums are not written.
    float2 xt[2], yt[2], zt[2], ltx[2], lty[2], ltz[2], ax[2], ay[2], az[2], cx[2], cy[2], cz[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int ta = tbase + threadIdx.x + 256 * p, tb = ta + 128;
        const long long ga = b0 + min(ta, ns - 1), gb = b0 + min(tb, ns - 1);
        const float4 pa = spos[ga], pb = spos[gb];
        const float4 la1 = sdup[3 * ga + 1], la2 = sdup[3 * ga + 2], lb1 = sdup[3 * gb + 1], lb2 = sdup[3 * gb + 2];
        const float ma = ta < ns ? 1.f : 0.f, mb = tb < ns ? 1.f : 0.f;
        xt[p] = make_float2(pa.x, pb.x);
        yt[p] = make_float2(pa.y, pb.y);
        zt[p] = make_float2(pa.z, pb.z);
        ltx[p] = make_float2(ma * la1.z, mb * lb1.z);
        lty[p] = make_float2(ma * la2.x, mb * lb2.x);
        ltz[p] = make_float2(ma * la2.z, mb * lb2.z);
        ax[p] = ay[p] = az[p] = cx[p] = cy[p] = cz[p] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    unsigned phase = 0;
    for (int J = it.J0; J < it.J1; ++J) {
        const int j0 = J * SYM_TILE;
        const int n = min(SYM_TILE, ns - j0);
        const int nr = (n + 31) & ~31;
        if (threadIdx.x == 0) {
            // the previous tile's generic-proxy reads and writes of sh are ordered before this copy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bulk_tile_load(sh, sdup + 3 * (b0 + j0), 48u * (unsigned)n, mbar);
        }
        const bool ok = mbar_wait(mbar, phase, first_polls);
        phase ^= 1u;
        // sources past the end of the suspension: position 0, lambda 0 (they add nothing)
        for (int e = n + threadIdx.x; e < nr; e += 128)
            sh[3 * e] = sh[3 * e + 1] = sh[3 * e + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(status + 1, 1);
                mbar_wait(mbar, phase ^ 1u);   // the copy in flight
            }
            return;
        }
        if (J == it.I) {
            // diagonal tile: every ordered pair, target side only (as the ordered kernel)
            for (int jc = 0; jc < nr; jc += 32) {
                float2 qx[2], qy[2], qz[2];
#pragma unroll
                for (int p = 0; p < 2; ++p) qx[p] = qy[p] = qz[p] = make_float2(0.f, 0.f);
#pragma unroll 4
                for (int j = jc; j < jc + 32; ++j) {
                    const float4 s0 = sh[3 * j], s1 = sh[3 * j + 1], s2 = sh[3 * j + 2];
                    const float2 xs = make_float2(s0.x, s0.y), ys = make_float2(s0.z, s0.w), zs = make_float2(s1.x, s1.y);
                    const float2 lx = make_float2(s1.z, s1.w), ly = make_float2(s2.x, s2.y), lz = make_float2(s2.z, s2.w);
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
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
                for (int p = 0; p < 2; ++p) {   // compensated addition of the sub-chunk sums
                    float2 y, u;
                    y = sub2(qx[p], cx[p]); u = add2(ax[p], y); cx[p] = sub2(sub2(u, ax[p]), y); ax[p] = u;
                    y = sub2(qy[p], cy[p]); u = add2(ay[p], y); cy[p] = sub2(sub2(u, ay[p]), y); ay[p] = u;
                    y = sub2(qz[p], cz[p]); u = add2(az[p], y); cz[p] = sub2(sub2(u, az[p]), y); az[p] = u;
                }
            }
        } else {
            for (int jc = 0; jc < nr; jc += 32) {
                float2 qx[2], qy[2], qz[2];
#pragma unroll
                for (int p = 0; p < 2; ++p) qx[p] = qy[p] = qz[p] = make_float2(0.f, 0.f);
                float2 jx = make_float2(0.f, 0.f), jy = jx, jz = jx;   // sums of the source this lane holds
#pragma unroll
                for (int st = 0; st < 32; ++st) {
                    const int j = jc + ((lane + st) & 31);
                    const float4 s0 = sh[3 * j], s1 = sh[3 * j + 1], s2 = sh[3 * j + 2];
                    const float2 xs = make_float2(s0.x, s0.y), ys = make_float2(s0.z, s0.w), zs = make_float2(s1.x, s1.y);
                    const float2 lx = make_float2(s1.z, s1.w), ly = make_float2(s2.x, s2.y), lz = make_float2(s2.z, s2.w);
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const float2 dx = sub2(xs, xt[p]), dy = sub2(ys, yt[p]), dz = sub2(zs, zt[p]);
                        const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
                        const float2 ri = make_float2(rsqrtf(fmaxf(r2.x, four_a2)), rsqrtf(fmaxf(r2.y, four_a2)));
                        const float2 ri2 = mul2(ri, ri);
                        const float2 ri3 = mul2(ri2, ri);
                        const float2 A = fma2(c23, ri3, ri);
                        const float2 B = mul2(ri3, fma2(mc2, ri2, one));
                        // target side: M lambda_source
                        const float2 s = mul2(B, fma2(dx, lx, fma2(dy, ly, mul2(dz, lz))));
                        qx[p] = fma2(A, lx, fma2(s, dx, qx[p]));
                        qy[p] = fma2(A, ly, fma2(s, dy, qy[p]));
                        qz[p] = fma2(A, lz, fma2(s, dz, qz[p]));
                        // source side: M lambda_target (the two halves are two targets)
                        const float2 w = mul2(B, fma2(dx, ltx[p], fma2(dy, lty[p], mul2(dz, ltz[p]))));
                        jx = fma2(A, ltx[p], fma2(w, dx, jx));
                        jy = fma2(A, lty[p], fma2(w, dy, jy));
                        jz = fma2(A, ltz[p], fma2(w, dz, jz));
                    }
                    // the source of lane l + 1 is lane l's next one
                    const int from = (lane + 1) & 31;
                    jx = shfl2(jx, from);
                    jy = shfl2(jy, from);
                    jz = shfl2(jz, from);
                }
                // after 32 passes the accumulator of source jc + lane is back at lane
                jsx[warp * SYM_TILE + jc + lane] = jx.x + jx.y;
                jsy[warp * SYM_TILE + jc + lane] = jy.x + jy.y;
                jsz[warp * SYM_TILE + jc + lane] = jz.x + jz.y;
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    float2 y, u;
                    y = sub2(qx[p], cx[p]); u = add2(ax[p], y); cx[p] = sub2(sub2(u, ax[p]), y); ax[p] = u;
                    y = sub2(qy[p], cy[p]); u = add2(ay[p], y); cy[p] = sub2(sub2(u, ay[p]), y); ay[p] = u;
                    y = sub2(qz[p], cz[p]); u = add2(az[p], y); cz[p] = sub2(sub2(u, az[p]), y); az[p] = u;
                }
            }
            __syncthreads();
            // the four warps' source-side sums, in warp order, into the (I, J) slot
            const long long slot = jbase[it.s] + (long long)J * (J - 1) / 2 + it.I;
            for (int e = threadIdx.x; e < n; e += 128) {
                const float sx = ((jsx[e] + jsx[SYM_TILE + e]) + jsx[2 * SYM_TILE + e]) + jsx[3 * SYM_TILE + e];
                const float sy = ((jsy[e] + jsy[SYM_TILE + e]) + jsy[2 * SYM_TILE + e]) + jsy[3 * SYM_TILE + e];
                const float sz = ((jsz[e] + jsz[SYM_TILE + e]) + jsz[2 * SYM_TILE + e]) + jsz[3 * SYM_TILE + e];
                part_j[slot * SYM_TILE + e] = make_float4(sx, sy, sz, 0.f);
            }
        }
        __syncthreads();   // sh and the sums are rewritten for the next tile
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float2 rx = sub2(ax[p], cx[p]), ry = sub2(ay[p], cy[p]), rz = sub2(az[p], cz[p]);
        const int ta = tbase + threadIdx.x + 256 * p, tb = ta + 128;
        if (ta < ns) part_i[(long long)it.k * NBL + b0 + ta] = make_float4(rx.x, ry.x, rz.x, 0.f);
        if (tb < ns) part_i[(long long)it.k * NBL + b0 + tb] = make_float4(rx.y, ry.y, rz.y, 0.f);
    }
}

// Work list: per suspension, T = ceil(n / SYM_TILE) tiles; row I holds tiles I..T-1, cut
// into items of at most `width` tiles (the first of a row holds the diagonal).  Fills the
// per-tile item counts (i-side slots), the per-suspension first j-side slot, and orders
// the items largest first.
void build_sym_list(const gdc_ctx* c, int width, std::vector<SymItem>& items, std::vector<int>& row_nk, int& kmax) {
    items.clear();
    row_nk.clear();
    kmax = 1;
    for (int s = 0; s < c->S; ++s) {
        const long long n = c->h_blob_off[s + 1] - c->h_blob_off[s];
        const int T = (int)((n + SYM_TILE - 1) / SYM_TILE);
        for (int I = 0; I < T; ++I) {
            int kk = 0;
            for (int J0 = I; J0 < T; J0 += width, ++kk) {
                SymItem it{};
                it.s = s;
                it.I = I;
                it.J0 = J0;
                it.J1 = std::min(T, J0 + width);
                it.k = kk;
                items.push_back(it);
            }
            row_nk.push_back(kk);
            kmax = std::max(kmax, kk);
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const SymItem& x, const SymItem& y) { return x.J1 - x.J0 > y.J1 - y.J0; });
}

void build_sym_items(gdc_ctx* c, int width) {
    c->sym_width = width;
    build_sym_list(c, width, c->h_sym_items, c->h_sym_row_nk, c->sym_kmax);
    c->h_sym_tile_base.assign(c->S + 1, 0);
    c->h_sym_jbase.assign(c->S + 1, 0);
    for (int s = 0; s < c->S; ++s) {
        const long long n = c->h_blob_off[s + 1] - c->h_blob_off[s];
        const int T = (int)((n + SYM_TILE - 1) / SYM_TILE);
        c->h_sym_tile_base[s + 1] = c->h_sym_tile_base[s] + T;
        c->h_sym_jbase[s + 1] = c->h_sym_jbase[s] + (long long)T * (T - 1) / 2;
    }
    c->sym_n_items = (int)c->h_sym_items.size();
}

gdc_status sym_upload(gdc_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->sym_items, c->h_sym_items.data(), sizeof(SymItem) * c->h_sym_items.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->sym_row_nk, c->h_sym_row_nk.data(), sizeof(int) * c->h_sym_row_nk.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->sym_tile_base, c->h_sym_tile_base.data(), sizeof(long long) * c->h_sym_tile_base.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->sym_jbase, c->h_sym_jbase.data(), sizeof(long long) * c->h_sym_jbase.size(),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "upload of the symmetric work list");
}

gdc_status sym_init_attributes(gdc_ctx* c) {
    cudaError_t e = cudaFuncSetAttribute(k_rpy32_sym<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SYM_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rpy32_sym<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, SYM_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rpy32_sym<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, SYM_SMEM);
    return cuda_check(c, e, "symmetric pair kernel attributes");
}

void launch_rpy32_sym(gdc_ctx* c) {
#define GDC_SYM_LAUNCH(MB)                                                                                         \
    k_rpy32_sym<MB><<<c->sym_n_items, 128, SYM_SMEM, c->stream>>>(c->sym_items, c->mv_active, c->susp_blob_off,     \
                                                                  c->sym_jbase, c->spos, c->sdup, c->sym_part_i,   \
                                                                  c->sym_part_j, c->NBL, rpy_const32(c->p.a),      \
                                                                  c->dev_status, first_wait_polls())
    ++c->n_launch;
    if (c->sym_minb == 3)
        GDC_SYM_LAUNCH(3);
    else if (c->sym_minb == 4)
        GDC_SYM_LAUNCH(4);
    else
        GDC_SYM_LAUNCH(2);
#undef GDC_SYM_LAUNCH
}

}  // namespace gdc
