// Symmetric double-float RPY pair kernel: the accurate residual product of the FP32-mixed
// mobility solve with every unordered pair of different bodies evaluated once for both of
// its blobs (M_ij = M_ji, even in d = r_j - r_i).  The pair's distance, reciprocal square
// root and coefficients A, B (about half its double-float operations) are shared; only the
// two products with lambda_j and lambda_i remain per side.
//
// Layout as in the symmetric FP32 kernel (sym.cu): tiles of 512 blobs; a block takes target
// tile I against source tiles J0..J1-1 (J >= I), the diagonal tile J = I ordered.  For J > I
// each warp holds 128 targets (four per lane); a 32-source sub-chunk is swept in 32 steps in
// which lane l takes source (l + step) mod 32, and the source-side sums (double-float) move
// one lane per step by shuffles, back at their source's lane after 32 steps.  At the end of
// each sub-chunk the four warps' source-side sums meet in shared memory (double-buffered, one
// barrier per sub-chunk) and warp 0 adds them in warp order into the tile pair's FP64 slot
// (deterministic).
// Target-side sums go to one FP64 slot per item.  Same-body pairs are skipped (the same-body
// block is added exactly in FP64 elsewhere).  Pairs are evaluated exactly as the ordered
// double-float kernel evaluates them (overlapping branch below 2a included).
#include <algorithm>

#include "common.cuh"
#include "df.cuh"

namespace gdc {

constexpr int DFS_TILE = GDC_SYM_TILE;
// dynamic shared memory: the source tile (four planes of one float4 per source: the lanes'
// rotated reads hit consecutive 16-byte words), then two buffers of the four
// warps' source sums of one 32-source sub-chunk (3 doubles per source each)
constexpr int DFS_SMEM = DFS_TILE * 4 * 16 + 2 * 4 * 3 * 32 * 8;

struct DfPair {   // the shared part of one pair: d = r_j - r_i, A, B
    df dx, dy, dz, A, B;
};

__device__ __forceinline__ DfPair df_pair(df xs, df ys, df zs, df xt, df yt, df zt, const RpyConstDF& k) {
    const df one{1.f, 0.f};
    DfPair p;
    p.dx = df_sub(xs, xt);
    p.dy = df_sub(ys, yt);
    p.dz = df_sub(zs, zt);
    const df r2 = df_add(df_add(df_mul(p.dx, p.dx), df_mul(p.dy, p.dy)), df_mul(p.dz, p.dz));
    const df ri = df_rsqrt(r2);
    if (r2.h > k.four_a2.h || (r2.h == k.four_a2.h && r2.l >= k.four_a2.l)) {
        const df ri2 = df_mul(ri, ri);
        const df ri3 = df_mul(ri2, ri);
        p.A = df_add(ri, df_mul(k.c23, ri3));
        p.B = df_mul(ri3, df_sub(one, df_mul(k.c2, ri2)));
    } else {   // overlapping blobs of different bodies (r > 0 for distinct blobs)
        const df r = df_mul(r2, ri);
        p.A = df_mul(k.cA, df_sub(one, df_mul(k.c9, r)));
        p.B = df_mul(k.cB, ri);
    }
    return p;
}

// u += A lambda + B (d . lambda) d
__device__ __forceinline__ void df_side(const DfPair& p, df lx, df ly, df lz, df& ux, df& uy, df& uz) {
    const df dl = df_add(df_add(df_mul(p.dx, lx), df_mul(p.dy, ly)), df_mul(p.dz, lz));
    const df s = df_mul(p.B, dl);
    ux = df_add(ux, df_add(df_mul(p.A, lx), df_mul(s, p.dx)));
    uy = df_add(uy, df_add(df_mul(p.A, ly), df_mul(s, p.dy)));
    uz = df_add(uz, df_add(df_mul(p.A, lz), df_mul(s, p.dz)));
}

__device__ __forceinline__ df shfl_df(df v, int src) {
    return df{__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src)};
}

// MINB: resident blocks per SM the register allocator is asked to allow, 3 (162 registers) or
// 4 (128); the autotuner times both against the ordered double-float kernel.
template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_rpy_df_sym(const SymItem* __restrict__ items,
                                                       const long long* __restrict__ susp_blob_off,
                                                       const long long* __restrict__ jbase,
                                                       const double4_32a* __restrict__ spos,
                                                       const double4_32a* __restrict__ slam,
                                                       double4_32a* __restrict__ part_i, double4_32a* __restrict__ part_j,
                                                       int NBL, RpyConstDF k) {
    extern __shared__ __align__(16) unsigned char dfs_smem[];
    float4* sh = reinterpret_cast<float4*>(dfs_smem);                       // [plane][source]
    double* ws = reinterpret_cast<double*>(dfs_smem + DFS_TILE * 4 * 16);  // [buffer][warp][3][32]
    const SymItem it = items[blockIdx.x];
    const long long b0 = susp_blob_off[it.s];
    const int ns = (int)(susp_blob_off[it.s + 1] - b0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tbase = it.I * DFS_TILE;
    // targets tbase + threadIdx.x + 128 m; a target past the end sits on the last blob with
    // lambda = 0 and body -1 (it adds nothing and its sums are not written)
    df xt[4], yt[4], zt[4], lxt[4], lyt[4], lzt[4], ux[4], uy[4], uz[4];
    float bt[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int t = tbase + threadIdx.x + 128 * m;
        const long long g = b0 + min(t, ns - 1);
        const double4_32a p = spos[g], l = slam[g];
        const bool in = t < ns;
        xt[m] = df_from(p.x);
        yt[m] = df_from(p.y);
        zt[m] = df_from(p.z);
        lxt[m] = df_from(in ? l.x : 0.0);
        lyt[m] = df_from(in ? l.y : 0.0);
        lzt[m] = df_from(in ? l.z : 0.0);
        bt[m] = in ? (float)p.w : -1.f;
        ux[m] = uy[m] = uz[m] = df{0.f, 0.f};
    }
    for (int J = it.J0; J < it.J1; ++J) {
        const int j0 = J * DFS_TILE;
        const int n = min(DFS_TILE, ns - j0);
        const int nr = (n + 31) & ~31;
        __syncthreads();   // the previous tile's sources and sums are no longer read
        for (int e = threadIdx.x; e < nr; e += 128) {
            if (e < n) {
                const double4_32a ps = spos[b0 + j0 + e], ls = slam[b0 + j0 + e];
                const df x = df_from(ps.x), y = df_from(ps.y), z = df_from(ps.z);
                const df lx = df_from(ls.x), ly = df_from(ls.y), lz = df_from(ls.z);
                sh[e] = make_float4(x.h, y.h, z.h, (float)ps.w);
                sh[DFS_TILE + e] = make_float4(x.l, y.l, z.l, 0.f);
                sh[2 * DFS_TILE + e] = make_float4(lx.h, ly.h, lz.h, 0.f);
                sh[3 * DFS_TILE + e] = make_float4(lx.l, ly.l, lz.l, 0.f);
            } else {   // padding: body -2 matches no target, lambda 0
                sh[e] = make_float4(0.f, 0.f, 0.f, -2.f);
                sh[DFS_TILE + e] = sh[2 * DFS_TILE + e] = sh[3 * DFS_TILE + e] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        if (J == it.I) {
            // diagonal tile: every ordered pair of different bodies, target side only
            for (int j = 0; j < n; ++j) {
                const float4 s0 = sh[j], s1 = sh[DFS_TILE + j], s2 = sh[2 * DFS_TILE + j], s3 = sh[3 * DFS_TILE + j];
                const df lx{s2.x, s3.x}, ly{s2.y, s3.y}, lz{s2.z, s3.z};
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    if (s0.w == bt[m] || bt[m] < 0.f) continue;   // same body, or no target
                    const DfPair p = df_pair(df{s0.x, s1.x}, df{s0.y, s1.y}, df{s0.z, s1.z}, xt[m], yt[m], zt[m], k);
                    df_side(p, lx, ly, lz, ux[m], uy[m], uz[m]);
                }
            }
        } else {
            const long long slot = jbase[it.s] + (long long)J * (J - 1) / 2 + it.I;
            for (int jc = 0; jc < nr; jc += 32) {
                df jx{0.f, 0.f}, jy{0.f, 0.f}, jz{0.f, 0.f};   // sums of the source this lane holds
                for (int st = 0; st < 32; ++st) {
                    const int j = jc + ((lane + st) & 31);
                    const float4 s0 = sh[j], s1 = sh[DFS_TILE + j], s2 = sh[2 * DFS_TILE + j], s3 = sh[3 * DFS_TILE + j];
                    const df xs{s0.x, s1.x}, ys{s0.y, s1.y}, zs{s0.z, s1.z};
                    const df lx{s2.x, s3.x}, ly{s2.y, s3.y}, lz{s2.z, s3.z};
                    const bool pad = s0.w < -1.5f;   // past the end of the suspension
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        if (pad || s0.w == bt[m] || bt[m] < 0.f) continue;   // padding, same body, no target
                        const DfPair p = df_pair(xs, ys, zs, xt[m], yt[m], zt[m], k);
                        df_side(p, lx, ly, lz, ux[m], uy[m], uz[m]);          // target side: M lambda_j
                        df_side(p, lxt[m], lyt[m], lzt[m], jx, jy, jz);       // source side: M lambda_i
                    }
                    const int from = (lane + 1) & 31;   // the source of lane l + 1 is lane l's next
                    jx = shfl_df(jx, from);
                    jy = shfl_df(jy, from);
                    jz = shfl_df(jz, from);
                }
                // after 32 passes the sums of source jc + lane are back at lane; the buffer this
                // sub-chunk writes was last read by warp 0 before the previous barrier
                double* wb = ws + ((jc >> 5) & 1) * (4 * 3 * 32);
                wb[(warp * 3 + 0) * 32 + lane] = df_to(jx);
                wb[(warp * 3 + 1) * 32 + lane] = df_to(jy);
                wb[(warp * 3 + 2) * 32 + lane] = df_to(jz);
                __syncthreads();
                if (warp == 0 && jc + lane < n) {   // the four warps' sums, in warp order
                    double v[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        v[c] = ((wb[(0 * 3 + c) * 32 + lane] + wb[(1 * 3 + c) * 32 + lane]) +
                                wb[(2 * 3 + c) * 32 + lane]) + wb[(3 * 3 + c) * 32 + lane];
                    part_j[slot * DFS_TILE + jc + lane] = make_double4_32a(v[0], v[1], v[2], 0.0);
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int t = tbase + threadIdx.x + 128 * m;
        if (t < ns)
            part_i[(long long)it.k * NBL + b0 + t] = make_double4_32a(df_to(ux[m]), df_to(uy[m]), df_to(uz[m]), 0.0);
    }
}

// u_i = c0 (target-side slots of the blob's tile row + source-side slots of the tiles before
// it, added in FP64 in a fixed order) [- K V]; the same-body blocks are added afterwards.
__global__ void k_rpy_df_sym_epilogue(int NBL, const double4_32a* __restrict__ part_i,
                                      const double4_32a* __restrict__ part_j, const int* __restrict__ blob_susp,
                                      const long long* __restrict__ susp_blob_off, const int* __restrict__ row_nk,
                                      const long long* __restrict__ tile_base, const long long* __restrict__ jbase,
                                      double c0, const double* __restrict__ x, double* __restrict__ y, int gm_layout,
                                      const int* __restrict__ blob_gm, const int* __restrict__ body_gm,
                                      const int* __restrict__ blob_body, const double* __restrict__ r,
                                      const double* __restrict__ Yc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const int s = blob_susp[i];
    const long long loc = i - susp_blob_off[s];
    const int J = (int)(loc / DFS_TILE), e = (int)(loc % DFS_TILE);
    const int n = row_nk[tile_base[s] + J];
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int kk = 0; kk < n; ++kk) {
        const double4_32a v = part_i[(long long)kk * NBL + i];
        ux += v.x;
        uy += v.y;
        uz += v.z;
    }
    const long long s0 = jbase[s] + (long long)J * (J - 1) / 2;
    for (int I = 0; I < J; ++I) {
        const double4_32a v = part_j[(s0 + I) * DFS_TILE + e];
        ux += v.x;
        uy += v.y;
        uz += v.z;
    }
    ux *= c0;
    uy *= c0;
    uz *= c0;
    if (!gm_layout) {
        y[3LL * i] = ux;
        y[3LL * i + 1] = uy;
        y[3LL * i + 2] = uz;
        return;
    }
    // saddle operator: M lambda - K V, K V = U_p + Omega_p x (r_i - Y_p)  (Eq. rigid_body_cond)
    const int p = blob_body[i];
    const double* V = x + body_gm[p];
    const double dx = r[3LL * i] - Yc[3 * p], dy = r[3LL * i + 1] - Yc[3 * p + 1], dz = r[3LL * i + 2] - Yc[3 * p + 2];
    const long long o = blob_gm[i];
    y[o] = ux - (V[0] + (V[4] * dz - V[5] * dy));
    y[o + 1] = uy - (V[1] + (V[5] * dx - V[3] * dz));
    y[o + 2] = uz - (V[2] + (V[3] * dy - V[4] * dx));
}

gdc_status dfsym_init_attributes(gdc_ctx* c) {
    cudaError_t e = cudaFuncSetAttribute(k_rpy_df_sym<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, DFS_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rpy_df_sym<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, DFS_SMEM);
    return cuda_check(c, e, "symmetric double-float kernel attributes");
}

// The symmetric double-float pair kernel alone (same-body blocks excluded).
void launch_rpy_df_sym_pairs(gdc_ctx* c) {
    ++c->n_launch;
    if (c->dfs_minb == 3)
        k_rpy_df_sym<3><<<c->dfs_n_items, 128, DFS_SMEM, c->stream>>>(c->dfs_items, c->susp_blob_off, c->sym_jbase,
                                                                       c->spos64, c->slam64, c->dfs_part_i,
                                                                       c->dfs_part_j, c->NBL, df_constants(c->p.a));
    else
        k_rpy_df_sym<4><<<c->dfs_n_items, 128, DFS_SMEM, c->stream>>>(c->dfs_items, c->susp_blob_off, c->sym_jbase,
                                                                       c->spos64, c->slam64, c->dfs_part_i,
                                                                       c->dfs_part_j, c->NBL, df_constants(c->p.a));
}

// Its epilogue: the slots into y (same-body blocks excluded; they are added afterwards).
void launch_rpy_df_sym_epilogue(gdc_ctx* c, const double* x, double* y, int gm_layout) {
    ++c->n_launch, k_rpy_df_sym_epilogue<<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(
        c->NBL, c->dfs_part_i, c->dfs_part_j, c->blob_susp, c->susp_blob_off, c->dfs_row_nk, c->sym_tile_base,
        c->sym_jbase, 1.0 / (8.0 * 3.141592653589793 * c->p.eta), x, y, gm_layout, c->blob_gm, c->body_gm,
        c->blob_body, c->r, c->Yc);
}

}  // namespace gdc
