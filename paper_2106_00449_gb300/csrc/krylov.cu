// Batched Krylov solvers of the mobility problem (Sec. 2.2): right-preconditioned
// GMRES on the saddle-point system of Eq. (lin_sys_RMB) with the block-diagonal P, and the
// Lanczos approximation of M^(1/2) W (Sec. 4.1, Chow & Saad).  Every suspension has its
// own Krylov space; vectors of all suspensions are stored back to back and reductions
// are segmented per suspension.  Reductions are two-pass (per-chunk partials, then a
// fixed-order sum per segment), so results are bitwise reproducible run to run.
//
// Precision: bases, inner products, Givens/Hessenberg and the square root of the small
// tridiagonal matrix of Lanczos are FP64 (at loose tolerances the stopping test alone runs
// on FP32 eigen-steps).  In
// GDC_FP32_MIXED mode the operator inside the Krylov loop uses the FP32 pair kernel; each
// GMRES cycle ends with an accurate residual (double-float pairs, FP64 same-body blocks),
// and the solver restarts from it until that residual meets gmres_tol (iterative refinement).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace gdc {

constexpr int RED_CHUNK = 1024;   // elements per reduction chunk
// FP32-mixed refinement: once every suspension's relative residual is at most this, the next
// residual is updated with the FP32 product of the (small) correction instead of recomputed
#define GDC_RESID_UPDATE 1e-3

// ---- segment / chunk tables ---------------------------------------------------------

static void build_seg(gdc::Seg& sg, const std::vector<long long>& off) {
    sg.h_off = off;
    sg.n = off.back();
    sg.h_chunks.clear();
    sg.h_seg_chunk_off.assign(off.size(), 0);
    for (size_t s = 0; s + 1 < off.size(); ++s) {
        sg.h_seg_chunk_off[s] = (int)sg.h_chunks.size();
        for (long long lo = off[s]; lo < off[s + 1]; lo += RED_CHUNK) {
            Chunk ch{};
            ch.lo = lo;
            ch.hi = std::min(off[s + 1], lo + RED_CHUNK);
            ch.seg = (int)s;
            sg.h_chunks.push_back(ch);
        }
    }
    sg.h_seg_chunk_off.back() = (int)sg.h_chunks.size();
    sg.n_chunks = (int)sg.h_chunks.size();
}

void setup_segments(gdc_ctx* c) {
    build_seg(c->seg_gm, c->h_gm_off);
    std::vector<long long> lz(c->S + 1);
    for (int s = 0; s <= c->S; ++s) lz[s] = 3 * c->h_blob_off[s];
    build_seg(c->seg_lz, lz);
}

// ---- reduction kernels -----------------------------------------------------------------

// part[chunk * cols + i] = sum over the chunk of V_i[e] * w[e], i < k  (V_i = V + i * ld)
//
// GB300 issues FP64 FMAs at a small fraction of its FP32 rate, so this kernel is bound by
// the FP64 pipe, not by HBM: each element of V costs one FMA.  A chunk is taken by two
// warps with 16 elements per lane, so the per-column warp reduction (5 shuffled adds)
// is small against the 16 FMAs per lane it follows; blockIdx.y takes MD_COLS columns, so
// that short vectors still give enough blocks.
// When kdev is given (graph mode) the count is k + *kdev: the loop index lives in device memory.
constexpr int MD_THREADS = 64;
constexpr int MD_PER = RED_CHUNK / MD_THREADS;
constexpr int MD_COLS = 8;

__global__ void __launch_bounds__(MD_THREADS) k_mdot(const Chunk* __restrict__ chunks, const double* __restrict__ V,
                                                     long long ld, int k, const int* __restrict__ kdev,
                                                     const double* __restrict__ w, double* __restrict__ part,
                                                     int cols) {
    __shared__ double sh[MD_THREADS / 32][MD_COLS];
    if (kdev) k += *kdev;
    const int i0 = blockIdx.y * MD_COLS;
    if (i0 >= k) return;
    const int i1 = min(k, i0 + MD_COLS);
    const Chunk ch = chunks[blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long e0 = ch.lo + threadIdx.x;
    const bool full = ch.hi - ch.lo == RED_CHUNK;
    double wv[MD_PER];
#pragma unroll
    for (int u = 0; u < MD_PER; ++u) {
        const long long e = e0 + u * MD_THREADS;
        wv[u] = e < ch.hi ? w[e] : 0.0;
    }
    for (int i = i0; i < i1; ++i) {
        const double* Vi = V + (long long)i * ld + e0;
        double a0 = 0.0, a1 = 0.0;
        if (full) {
#pragma unroll
            for (int u = 0; u < MD_PER; u += 2) {
                a0 = fma(Vi[u * MD_THREADS], wv[u], a0);
                a1 = fma(Vi[(u + 1) * MD_THREADS], wv[u + 1], a1);
            }
        } else {
#pragma unroll
            for (int u = 0; u < MD_PER; u += 2) {
                if (e0 + u * MD_THREADS < ch.hi) a0 = fma(Vi[u * MD_THREADS], wv[u], a0);
                if (e0 + (u + 1) * MD_THREADS < ch.hi) a1 = fma(Vi[(u + 1) * MD_THREADS], wv[u + 1], a1);
            }
        }
        const double acc = warp_sum(a0 + a1);
        if (lane == 0) sh[wid][i - i0] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < i1 - i0; i += blockDim.x)
        part[(long long)blockIdx.x * cols + i0 + i] = sh[0][i] + sh[1][i];
}

// out[s * cols + i] = sum of the chunk partials of segment s, in chunk order
// One warp per (segment, column): lanes take chunks lane, lane+32, ... and the warp sums
// them with a fixed shuffle tree, so the order is the same on every run.
__global__ void k_seg_sum(int S, const int* __restrict__ seg_chunk_off, const double* __restrict__ part, int cols, int k,
                          const int* __restrict__ kdev, double* __restrict__ out) {
    if (kdev) k += *kdev;
    const int s = blockIdx.x;
    const int i = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= k) return;
    double acc = 0.0;
    for (int ch = seg_chunk_off[s] + lane; ch < seg_chunk_off[s + 1]; ch += 32) acc += part[(long long)ch * cols + i];
    acc = warp_sum(acc);
    if (lane == 0) out[(long long)s * cols + i] = acc;
}

// w[e] -= sum_i h[s * cols + i] * V_i[e] for i < k   (FP64-pipe bound like k_mdot; each thread
// updates its four elements together so that four loads and FMAs are in flight per column)
__global__ void __launch_bounds__(256) k_mupdate(const Chunk* __restrict__ chunks, const double* __restrict__ V,
                                                 long long ld, int k, const int* __restrict__ kdev,
                                                 const double* __restrict__ h, int cols, double* __restrict__ w) {
    if (kdev) k += *kdev;
    const Chunk ch = chunks[blockIdx.x];
    const double* hs = h + (long long)ch.seg * cols;
    constexpr int PER = RED_CHUNK / 256;
    const long long e0 = ch.lo + threadIdx.x;
    double acc[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const long long e = e0 + u * 256;
        acc[u] = e < ch.hi ? w[e] : 0.0;
    }
    for (int i = 0; i < k; ++i) {
        const double hv = -hs[i];
        const double* Vi = V + (long long)i * ld + e0;
#pragma unroll
        for (int u = 0; u < PER; ++u)
            if (e0 + u * 256 < ch.hi) acc[u] = fma(hv, Vi[u * 256], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u)
        if (e0 + u * 256 < ch.hi) w[e0 + u * 256] = acc[u];
}

// out[e] = scale_s * sum_i y[s * cols + i] * V_i[e] for i < kcount[s]   (+ out[e] when accumulate)
__global__ void k_combine(const Chunk* __restrict__ chunks, const double* __restrict__ V, long long ld,
                          const int* __restrict__ kcount, const double* __restrict__ y, int cols,
                          const double* __restrict__ scale, double* __restrict__ out) {
    const Chunk ch = chunks[blockIdx.x];
    const int k = kcount[ch.seg];
    const double* ys = y + (long long)ch.seg * cols;
    const double sc = scale ? scale[ch.seg] : 1.0;
    for (long long e = ch.lo + threadIdx.x; e < ch.hi; e += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc = fma(ys[i], V[(long long)i * ld + e], acc);
        out[e] = sc * acc;
    }
}

// out[e] = w[e] * scal[s]
__global__ void k_seg_scale(const Chunk* __restrict__ chunks, const double* __restrict__ w,
                            const double* __restrict__ scal, double* __restrict__ out) {
    const Chunk ch = chunks[blockIdx.x];
    const double sc = scal[ch.seg];
    for (long long e = ch.lo + threadIdx.x; e < ch.hi; e += blockDim.x) out[e] = w[e] * sc;
}

// out_base + (jadd + *jdev) * ld  <-  w * scal[s]   (and a copy into also, when given)
__global__ void k_seg_scale_slot(const Chunk* __restrict__ chunks, const double* __restrict__ w,
                                 const double* __restrict__ scal, double* __restrict__ out_base, long long ld,
                                 const int* __restrict__ jdev, int jadd, double* __restrict__ also) {
    const Chunk ch = chunks[blockIdx.x];
    const double sc = scal[ch.seg];
    double* out = out_base + (long long)(jadd + (jdev ? *jdev : 0)) * ld;
    for (long long e = ch.lo + threadIdx.x; e < ch.hi; e += blockDim.x) {
        const double v = w[e] * sc;
        out[e] = v;
        if (also) also[e] = v;
    }
}

__global__ void k_axpy_chunks(const Chunk* __restrict__ chunks, double a, const double* __restrict__ x,
                              double* __restrict__ y) {
    const Chunk ch = chunks[blockIdx.x];
    for (long long e = ch.lo + threadIdx.x; e < ch.hi; e += blockDim.x) y[e] += a * x[e];
}

__global__ void k_sub_chunks(const Chunk* __restrict__ chunks, const double* __restrict__ b,
                             const double* __restrict__ ax, double* __restrict__ r) {
    const Chunk ch = chunks[blockIdx.x];
    for (long long e = ch.lo + threadIdx.x; e < ch.hi; e += blockDim.x) r[e] = b[e] - ax[e];
}

// per-segment inner products <V_i, w>, i < k  -> out[s * cols + i]
// kdev (graph mode): the count is k + *kdev, at most kcap; the column grid covers kcap
static void seg_mdot(gdc_ctx* c, const gdc::Seg& sg, const double* V, long long ld, int k, const double* w,
                     double* out, int cols, const int* kdev = nullptr, int kcap = 0) {
    ++c->n_launch, k_mdot<<<dim3(sg.n_chunks, ceil_div(kdev ? kcap : k, MD_COLS)), MD_THREADS, 0, c->stream>>>(
        sg.chunks, V, ld, k, kdev, w, c->red_part, c->red_cols);
    ++c->n_launch, k_seg_sum<<<dim3(c->S, ceil_div(kdev ? kcap : k, 8)), 256, 0, c->stream>>>(
        c->S, sg.seg_chunk_off, c->red_part, c->red_cols, k, kdev, out);
    (void)cols;
}


// ---- tiny per-suspension helpers ------------------------------------------------------

__global__ void k_sqrt_col0(int S, const double* __restrict__ v, int cols, double* __restrict__ o) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) o[s] = sqrt(fmax(v[(long long)s * cols], 0.0));
}

__global__ void k_add_cols(int k, const int* __restrict__ kdev, double* __restrict__ h, const double* __restrict__ h2,
                           int cols) {
    if (kdev) k += *kdev;
    const int s = blockIdx.x;
    for (int i = threadIdx.x; i < k; i += blockDim.x) h[(long long)s * cols + i] += h2[(long long)s * cols + i];
}

__global__ void k_fill(int S, double v, double* __restrict__ o) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) o[s] = v;
}

// ---- operators ---------------------------------------------------------------------

gdc_status rpy_op(gdc_ctx* c, int prec, const double* lam, double* u) {
    if (c->fcm) {   // the periodic FCM mobility (one suspension, lambda and u 3 per blob)
        const gdc_status st = gdc_fcm_apply(c->fcm, (int)c->NBL, c->r, lam, u);
        return st == GDC_OK ? st : fail(c, st, std::string("FCM: ") + gdc_fcm_last_error(c->fcm));
    }
    launch_pack_lambda(c, prec, lam, 0);
    launch_rpy(c, prec);
    launch_rpy_epilogue(c, prec, lam, u, 0);
    if (c->p.wall) launch_wall_apply(c, prec, lam, u, 0);   // + the wall correction of every pair
    return GDC_OK;
}

gdc_status saddle_op(gdc_ctx* c, int prec, const double* x, double* y) {
    if (c->fcm) {   // one suspension: lambda is the first 3 N_b entries of the saddle vector
        const gdc_status st = gdc_fcm_apply(c->fcm, (int)c->NBL, c->r, x, c->fcm_u);
        if (st != GDC_OK) return fail(c, st, std::string("FCM: ") + gdc_fcm_last_error(c->fcm));
        launch_fcm_saddle_rows(c, x, y);
        launch_body_KT(c, x, 1, y, 1, -1.0);
        return GDC_OK;
    }
    launch_pack_lambda(c, prec, x, 1);
    launch_rpy(c, prec);
    launch_rpy_epilogue(c, prec, x, y, 1);
    if (c->p.wall) launch_wall_apply(c, prec, x, y, 1);
    launch_body_KT(c, x, 1, y, 1, -1.0);
    return GDC_OK;
}

// The operator whose Krylov space Lanczos builds (Sec. 4.1): M, or with lanczos_precond the
// block-preconditioned A = L^-1 M L^-T of Chow & Saad, L = diag_p(L_p) with L_p L_p^T = M_pp.
// Since L_p^-1 M_pp L_p^-T = I, an FP32 product takes A x = x + L^-1 M_off L^-T x with M_off
// the blocks between different bodies (the FP32 product without its same-body blocks), so
// the body blocks of A are the identity exactly; FP64, and every product above a wall (whose
// correction couples a body's blobs too), forms L^-1 (M (L^-T x)).
static void lz_operator(gdc_ctx* c, int prec, const double* x, double* w) {
    if (!c->p.lanczos_precond) {
        rpy_op(c, prec, x, w);
        return;
    }
    if (prec == GDC_FP32_MIXED && !c->p.wall) {
        // the factor products in FP32 too: the coupling term they feed carries FP32 rounding
        launch_body_tri(c, TRI_LINV_T, x, nullptr, c->lz_z, true);
        launch_pack_lambda(c, prec, c->lz_z, 0);
        launch_rpy(c, prec);
        launch_rpy_epilogue(c, prec, c->lz_z, c->lz_u, 0, false);
        launch_body_tri(c, TRI_LINV, c->lz_u, x, w, true);
    } else {
        launch_body_tri(c, TRI_LINV_T, x, nullptr, c->lz_z);
        rpy_op(c, prec, c->lz_z, c->lz_u);
        launch_body_tri(c, TRI_LINV, c->lz_u, nullptr, w);
    }
}

// out = scale * V c, and with lanczos_precond the factor L applied to it: L A^(1/2) W
static void lz_result(gdc_ctx* c, double scale, double* out) {
    const gdc::Seg& sg = c->seg_lz;
    const long long n = 3LL * c->NBL;
    double* comb = c->p.lanczos_precond ? c->lz_w : out;
    ++c->n_launch, k_fill<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, scale, c->lz_scal);
    ++c->n_launch, k_combine<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->lz_V, n, c->lz_k, c->lz_c, c->kmax,
                                                                 c->lz_scal, comb);
    if (c->p.lanczos_precond) launch_body_tri(c, TRI_L, comb, nullptr, out);
}

static gdc_status sync_read(gdc_ctx* c, const void* dev, void* host, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "device-to-host read");
}

// ---- GMRES small per-suspension kernels ------------------------------------------------

// Start of a cycle: beta = ||r||, residual check against tol, V_0 scale and g.
__global__ void k_gm_start(int S, const double* __restrict__ rn2, const double* __restrict__ bnorm, double tol,
                           int cols, double* __restrict__ res, int* __restrict__ active, double* __restrict__ g,
                           double* __restrict__ scal, int mp1, int* __restrict__ jcount, int* __restrict__ outer) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double beta = sqrt(fmax(rn2[(long long)s * cols], 0.0));
    const double bn = bnorm[s];
    const double rr = bn > 0.0 ? beta / bn : 0.0;
    res[s] = rr;
    const int go = (bn > 0.0) && (rr > tol) && isfinite(rr);
    outer[s] = go || !isfinite(rr);
    active[s] = go;
    jcount[s] = 0;
    for (int i = 0; i < mp1; ++i) g[(long long)s * mp1 + i] = 0.0;
    g[(long long)s * mp1] = beta;
    scal[s] = (go && beta > 0.0) ? 1.0 / beta : 0.0;
}

// Column j of the Hessenberg matrix: h (orthogonalisation coefficients), beta = ||w||.
// Applies the previous Givens rotations, makes a new one, updates g and the residual estimate.
__global__ void k_gm_arnoldi(int S, int j, const int* __restrict__ jdev, int m, const double* __restrict__ h, int cols,
                             const double* __restrict__ wn2, double* __restrict__ H, double* __restrict__ cs,
                             double* __restrict__ sn, double* __restrict__ g, const double* __restrict__ bnorm,
                             double inner_tol, double* __restrict__ est, int* __restrict__ active,
                             int* __restrict__ jcount, double* __restrict__ scal) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    if (jdev) j = *jdev;
    if (!active[s]) {
        scal[s] = 0.0;
        return;
    }
    const int mp1 = m + 1;
    double* Hs = H + (long long)s * mp1 * m;
    double* css = cs + (long long)s * m;
    double* sns = sn + (long long)s * m;
    double* gs = g + (long long)s * mp1;
    const double beta = sqrt(fmax(wn2[(long long)s * cols], 0.0));
    for (int i = 0; i <= j; ++i) Hs[i * m + j] = h[(long long)s * cols + i];
    Hs[(j + 1) * m + j] = beta;
    for (int i = 0; i < j; ++i) {
        const double a = Hs[i * m + j], b = Hs[(i + 1) * m + j];
        Hs[i * m + j] = css[i] * a + sns[i] * b;
        Hs[(i + 1) * m + j] = -sns[i] * a + css[i] * b;
    }
    const double a = Hs[j * m + j], b = Hs[(j + 1) * m + j];
    const double rr = hypot(a, b);
    const double cc = rr > 0.0 ? a / rr : 1.0, ss = rr > 0.0 ? b / rr : 0.0;
    css[j] = cc;
    sns[j] = ss;
    Hs[j * m + j] = rr;
    Hs[(j + 1) * m + j] = 0.0;
    gs[j + 1] = -ss * gs[j];
    gs[j] = cc * gs[j];
    const double e = fabs(gs[j + 1]) / bnorm[s];
    est[s] = e;
    jcount[s] = j + 1;
    scal[s] = beta > 0.0 ? 1.0 / beta : 0.0;
    if (!(e > inner_tol) || beta == 0.0 || j + 1 == m) active[s] = 0;
}

// y = H^-1 g (upper triangular, size jcount[s])
__global__ void k_gm_backsolve(int S, int m, const double* __restrict__ H, const double* __restrict__ g,
                               const int* __restrict__ jcount, double* __restrict__ y, int cols) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int k = jcount[s];
    const int mp1 = m + 1;
    const double* Hs = H + (long long)s * mp1 * m;
    const double* gs = g + (long long)s * mp1;
    double* ys = y + (long long)s * cols;
    for (int i = k - 1; i >= 0; --i) {
        double acc = gs[i];
        for (int q = i + 1; q < k; ++q) acc -= Hs[i * m + q] * ys[q];
        ys[i] = Hs[i * m + i] != 0.0 ? acc / Hs[i * m + i] : 0.0;
    }
    for (int i = k; i < cols; ++i) ys[i] = 0.0;
}

gdc_status gmres_solve(gdc_ctx* c, const double* b, double* x, gdc_solve_info* info) {
    // FCM: one operator whatever the precision, so no refinement against a second product
    const int prec = c->fcm ? GDC_FP64 : c->p.precision;
    const int m = c->m;
    const long long n = c->ngm;
    const gdc::Seg& sg = c->seg_gm;
    const int cols = c->red_cols;
    const double tol = c->p.gmres_tol;
    // the FP32 cycle aims below tol so that one FP64 residual usually confirms it
    const double inner_tol = prec == GDC_FP32_MIXED ? 0.1 * tol : tol;
    gdc_solve_info inf{};
    // ||b|| per suspension
    seg_mdot(c, sg, b, 0, 1, b, c->gm_h, cols);
    double* bn2 = c->gm_h;
    // bnorm = sqrt(bn2): reuse k_seg_scale-free path via a tiny kernel
    ++c->n_launch, k_sqrt_col0<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, bn2, cols, c->gm_bnorm);
    cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream);
    cudaMemcpyAsync(c->gm_r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream);
    int total = 0;
    gdc_status st = GDC_OK;
    std::vector<int> outer(c->S), act(c->S);
    std::vector<double> res(c->S);
    for (int cycle = 0;; ++cycle) {
        // beta = ||r|| and the FP64 residual check
        seg_mdot(c, sg, c->gm_r, 0, 1, c->gm_r, c->gm_h2, cols);
        ++c->n_launch, k_gm_start<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, c->gm_h2, c->gm_bnorm, tol, cols, c->gm_res,
                                                               c->gm_active, c->gm_g, c->gm_scal, m + 1, c->gm_j,
                                                               c->gm_active + c->S);
        if ((st = sync_read(c, c->gm_active + c->S, outer.data(), sizeof(int) * c->S)) != GDC_OK) return st;
        if ((st = sync_read(c, c->gm_res, res.data(), sizeof(double) * c->S)) != GDC_OK) return st;
        inf.cycles = cycle;
        double rmax = 0.0;
        bool any = false, bad = false;
        for (int s = 0; s < c->S; ++s) {
            if (!std::isfinite(res[s])) bad = true;
            rmax = std::max(rmax, res[s]);
            any = any || outer[s];
        }
        inf.residual = rmax;
        if (bad) {
            st = fail(c, GDC_ERR_NONFINITE, "mobility solve: non-finite residual");
            break;
        }
        if (!any) {
            inf.converged = 1;
            break;
        }
        if (total >= c->p.gmres_max_iter) {
            st = fail(c, GDC_ERR_NOT_CONVERGED, "mobility solve: GMRES reached gmres_max_iter");
            break;
        }
        ++c->n_launch, k_seg_scale<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_r, c->gm_scal, c->gm_V);
        int j = 0;
        for (; j < m; ++j) {
            double* Vj = c->gm_V + (long long)j * n;
            launch_precond(c, Vj, c->gm_z, prec == GDC_FP32_MIXED);
            c->mv_active = c->gm_active;   // suspensions that have converged need no product
            saddle_op(c, prec, c->gm_z, c->gm_w);
            c->mv_active = nullptr;
            if (prec == GDC_FP32_MIXED) inf.matvecs_fp32++; else inf.matvecs_fp64++;
            // classical Gram-Schmidt, twice
            seg_mdot(c, sg, c->gm_V, n, j + 1, c->gm_w, c->gm_h, cols);
            ++c->n_launch, k_mupdate<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_V, n, j + 1, nullptr, c->gm_h, cols, c->gm_w);
            seg_mdot(c, sg, c->gm_V, n, j + 1, c->gm_w, c->gm_h2, cols);
            ++c->n_launch, k_mupdate<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_V, n, j + 1, nullptr, c->gm_h2, cols, c->gm_w);
            ++c->n_launch, k_add_cols<<<c->S, 128, 0, c->stream>>>(j + 1, nullptr, c->gm_h, c->gm_h2, cols);
            // ||w||: the column of wn2 lives after the h coefficients
            seg_mdot(c, sg, c->gm_w, 0, 1, c->gm_w, c->gm_h2, cols);
            ++c->n_launch, k_gm_arnoldi<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, j, nullptr, m, c->gm_h, cols, c->gm_h2, c->gm_H,
                                                                     c->gm_cs, c->gm_sn, c->gm_g, c->gm_bnorm,
                                                                     inner_tol, c->gm_res + c->S, c->gm_active,
                                                                     c->gm_j, c->gm_scal);
            ++c->n_launch, k_seg_scale<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_w, c->gm_scal, c->gm_V + (long long)(j + 1) * n);
            ++total;
            if ((st = sync_read(c, c->gm_active, act.data(), sizeof(int) * c->S)) != GDC_OK) return st;
            bool still = false;
            for (int s = 0; s < c->S; ++s) still = still || act[s];
            if (!still || total >= c->p.gmres_max_iter) {
                ++j;
                break;
            }
        }
        inf.iterations = std::max(inf.iterations, total);
        // x += P^-1 V y
        ++c->n_launch, k_gm_backsolve<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, m, c->gm_H, c->gm_g, c->gm_j, c->gm_y, cols);
        ++c->n_launch, k_combine<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_V, n, c->gm_j, c->gm_y, cols, nullptr, c->gm_w);
        launch_precond(c, c->gm_w, c->gm_z, prec == GDC_FP32_MIXED);   // the correction e of this cycle
        ++c->n_launch, k_axpy_chunks<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, 1.0, c->gm_z, x);
        if (prec == GDC_FP32_MIXED && rmax <= GDC_RESID_UPDATE) {
            // r <- r - A e: the residual is already small, so A e is too, and the FP32 product's
            // relative error (~3e-7) leaves r accurate to ~3e-7 * rmax, far below gmres_tol
            saddle_op(c, GDC_FP32_MIXED, c->gm_z, c->gm_w);
            inf.matvecs_fp32++;
            ++c->n_launch, k_axpy_chunks<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, -1.0, c->gm_w, c->gm_r);
        } else {
            // accurate residual r = b - A x: FP64 in FP64 mode; double-float pairs + FP64
            // same-body blocks in mixed mode
            saddle_op(c, prec == GDC_FP32_MIXED ? GDC_PREC_DF64 : GDC_FP64, x, c->gm_w);
            inf.matvecs_fp64++;
            ++c->n_launch, k_sub_chunks<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, b, c->gm_w, c->gm_r);
        }
        if ((st = cuda_check(c, cudaGetLastError(), "GMRES launch")) != GDC_OK) return st;
    }
    inf.iterations = total;
    if (info) *info = inf;
    return st;
}

// ---- Lanczos square root ------------------------------------------------------------

__global__ void k_lz_start(int S, const double* __restrict__ wn2, int cols, double* __restrict__ Wnorm,
                           double* __restrict__ scal, int* __restrict__ active, int* __restrict__ kcount,
                           double* __restrict__ err) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double nrm = sqrt(fmax(wn2[(long long)s * cols], 0.0));
    Wnorm[s] = nrm;
    scal[s] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    active[s] = nrm > 0.0;
    kcount[s] = 0;
    err[s] = 0.0;
}

// Lanczos bookkeeping and, where needed, c = ||W|| T_k^(1/2) e_1 for one suspension
// (one warp per suspension).
//
// T_k = Q diag(theta) Q^T is diagonalised by implicit symmetric QR steps with
// Wilkinson shifts (Golub & Van Loan, Sec. 8.3).  Every lane runs the same sweep on its
// own copy of the diagonal and off-diagonal (identical arithmetic, so identical values and
// warp-uniform control flow); the bulge chase keeps its carried entries in registers, so
// the serial chain per rotation is one Givens rotation and a few fused multiply-adds.
// Q is accumulated in shared memory, each lane updating the rows it owns (rows lane,
// lane + 32, ...), off the serial chain.  Then c = wn Q (sqrt(theta) o Q^T e_1), where
// Q^T e_1 is row 0 of Q.
//
// Convergence: ||c_k - c_{k-1}|| / ||c_k|| < tol, evaluated from a start index set by the
// suspension's previous count (so early iterations skip the eigen-work);
// in fixed mode c is formed once, at k = fixed[s].
static_assert(GDC_MAX_LANCZOS <= 128, "a lane owns at most 4 rows of Q");

// Row stride of Q in shared memory: odd, so that the lanes' rows fall in distinct banks.
__host__ __device__ inline int lz_ldq(int kmax) { return kmax | 1; }

// The FP64 root at the stopping index is refined from the FP32 eigendecomposition up to
// this many Lanczos vectors (its scratch grows as k^2), formed by FP64 QR beyond.
#define GDC_LZ_REFINE_MAX 64

// Doubles of scratch the refined root needs for k vectors: Q in FP32, Z and W in FP64, two
// vectors (see lz_sqrt_e1_refined).
__host__ __device__ inline int lz_refine_doubles(int k) {
    const int ldk = k | 1;
    return (k * ldk + 1) / 2 + 2 * k * ldk + 2 * k;
}

__device__ inline long long lz_q_doubles_dev(int kmax) {
    const int q = kmax * lz_ldq(kmax), r = lz_refine_doubles(kmax < GDC_LZ_REFINE_MAX ? kmax : GDC_LZ_REFINE_MAX);
    return q > r ? q : r;
}

// Doubles of Q (FP64, or FP32 in half of them) or of the scratch of the refined root,
// whichever is larger.
long long lz_q_doubles(int kmax) {
    return std::max(kmax * lz_ldq(kmax), lz_refine_doubles(std::min(kmax, GDC_LZ_REFINE_MAX)));
}

// Dynamic shared memory of k_lz_tridiag: four c vectors, then Q or the refined root's scratch
// (132 KB at kmax = 128, one block per SM).  With more suspensions than SMs that area lives in
// a per-suspension slice of global memory instead (c->lz_qbuf, cached in L1), so that several
// suspensions' warps share an SM.
static size_t lz_tridiag_smem(int kmax) { return (size_t)(4 * kmax + lz_q_doubles(kmax)) * sizeof(double); }
static size_t lz_launch_smem(const gdc_ctx* c) {
    return c->lz_qbuf_on ? (size_t)4 * c->kmax * sizeof(double) : lz_tridiag_smem(c->kmax);
}

// Givens rotation (c, s) with c x + s z = r, -s x + c z = 0.  FP32 (the stopping test at
// loose tolerances) takes 1/r from the hardware reciprocal square root; FP64 divides by the
// correctly rounded square root.
__device__ inline void lz_givens(float x, float z, float& c, float& s, float& r) {
    const float r2 = fmaf(x, x, z * z);
    if (r2 > 0.f) {
        const float ri = rsqrtf(r2);
        c = x * ri;
        s = z * ri;
        r = r2 * ri;
    } else {
        c = 1.f;
        s = 0.f;
        r = 0.f;
    }
}
__device__ inline void lz_givens(double x, double z, double& c, double& s, double& r) {
    r = sqrt(x * x + z * z);
    if (r > 0.0) {
        const double ri = 1.0 / r;
        c = x * ri;
        s = z * ri;
    } else {
        c = 1.0;
        s = 0.0;
    }
}

// out[0..k) = wn * T_k^(1/2) e_1 for the k x k tridiagonal (al, be), computed in precision T
// by the whole warp; Q is k x k in shared memory with row stride ldq.  Returns false (on
// every lane) when the QR iteration does not converge.
template <typename T>
__device__ bool lz_sqrt_e1_t(const double* al, const double* be, int k, double wn, T* Q, int ldq, double* out) {
    const int lane = threadIdx.x;
    const T eps = sizeof(T) == 4 ? T(1.2e-7) : T(1e-16);   // deflation threshold (relative)
    T d[GDC_MAX_LANCZOS], e[GDC_MAX_LANCZOS];
    for (int i = 0; i < k; ++i) {
        d[i] = (T)al[i];
        e[i] = i + 1 < k ? (T)be[i] : T(0);
    }
    for (int r = lane; r < k; r += 32)
        for (int col = 0; col < k; ++col) Q[r * ldq + col] = r == col ? T(1) : T(0);
    int hi = k - 1;
    for (int sweep = 0; hi > 0; ++sweep) {
        if (sweep > 40 * k + 40) return false;
        if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
            e[hi - 1] = T(0);
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
        const T del = T(0.5) * (d[hi - 1] - d[hi]);
        const T bb = e[hi - 1];
        const T sg = del >= T(0) ? T(1) : T(-1);
        const T mu = d[hi] - bb * bb / (del + sg * sqrt(del * del + bb * bb));
        // carried: dq = d[q] and eq = e[q] as the previous rotation left them
        T dq = d[lo], eq = e[lo];
        T x = dq - mu, z = eq;
        T qc[4];   // column q of the lane's rows of Q
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int r = lane + 32 * m;
            qc[m] = r < k ? Q[r * ldq + lo] : T(0);
        }
        for (int q = lo; q < hi; ++q) {
            const T dq1 = d[q + 1];
            const T eq1 = q + 1 < hi ? e[q + 1] : T(0);
            T cq, sq, rr;
            lz_givens(x, z, cq, sq, rr);
            if (q > lo) e[q - 1] = rr;
            const T cc = cq * cq, ss = sq * sq, cs = cq * sq;
            d[q] = cc * dq + T(2) * cs * eq + ss * dq1;
            const T nd1 = ss * dq - T(2) * cs * eq + cc * dq1;
            const T ne = cs * (dq1 - dq) + (cc - ss) * eq;
            e[q] = ne;
            dq = nd1;
            x = ne;
            z = sq * eq1;
            eq = cq * eq1;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int r = lane + 32 * m;
                if (r < k) {
                    const T qn = Q[r * ldq + q + 1];
                    Q[r * ldq + q] = cq * qc[m] + sq * qn;
                    qc[m] = -sq * qc[m] + cq * qn;
                }
            }
        }
        d[hi] = dq;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int r = lane + 32 * m;
            if (r < k) Q[r * ldq + hi] = qc[m];
        }
    }
    __syncwarp();   // row 0 of Q (lane 0's) is read by every lane
    for (int i = 0; i < k; ++i) e[i] = sqrt(d[i] > T(0) ? d[i] : T(0)) * Q[i];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int r = lane + 32 * m;
        if (r < k) {
            T acc = T(0);
            for (int i = 0; i < k; ++i) acc += Q[r * ldq + i] * e[i];
            out[r] = wn * (double)acc;
        }
    }
    __syncwarp();   // out complete before any lane reads it, Q free for the next call
    return true;
}

// The square root that enters v-breve is always formed in FP64.  At loose tolerances
// (lanczos_tol >= 1e-5) the stopping test alone compares FP32 iterates: their relative
// error, about 1e-6, is far below the tolerance the change is compared with.
__device__ inline bool lz_sqrt_e1(const double* al, const double* be, int k, double wn, double* Q, int ldq, double* out,
                                  bool fp32) {
    return fp32 ? lz_sqrt_e1_t<float>(al, be, k, wn, reinterpret_cast<float*>(Q), ldq, out)
                : lz_sqrt_e1_t<double>(al, be, k, wn, Q, ldq, out);
}

// out = wn T^(1/2) e_1 in FP64 from the FP32 eigendecomposition T ~ Q diag(theta) Q^T, refined
// once (k <= GDC_LZ_REFINE_MAX): Z = Q (3I - Q^T Q)/2 is orthogonal to O(|Q^T Q - I|^2), and
// in B = Z^T T Z = D + E (D its diagonal, E of the size of the FP32 rounding) the root
// X = D^(1/2) + Y with Y_ij = E_ij / (sqrt(d_i) + sqrt(d_j)) satisfies X^2 = B + O(|E|^2),
// so T^(1/2) e_1 = Z X Z^T e_1 to about 1e-12 relative.  The denominators are sums of square
// roots, never small differences, so close eigenvalues are no difficulty.  All sums in FP64,
// spread over the warp.  buf holds lz_refine_doubles(k) doubles.
__device__ bool lz_sqrt_e1_refined(const double* al, const double* be, int k, double wn, double* buf, double* out) {
    const int lane = threadIdx.x, ldk = k | 1;
    float* Qf = reinterpret_cast<float*>(buf);
    double* Z = buf + (k * ldk + 1) / 2;
    double* Wm = Z + k * ldk;
    double* sv = Wm + k * ldk;   // sqrt(d_j)
    double* hv = sv + k;         // X Z^T e_1
    if (!lz_sqrt_e1_t<float>(al, be, k, wn, Qf, ldk, out)) return false;
    // G = Q^T Q into Wm
    for (int e = lane; e < k * k; e += 32) {
        const int i = e / k, j = e % k;
        double acc = 0.0;
        for (int r = 0; r < k; ++r) acc = fma((double)Qf[r * ldk + i], (double)Qf[r * ldk + j], acc);
        Wm[i * ldk + j] = acc;
    }
    __syncwarp();
    // Z = Q (3I - G) / 2
    for (int e = lane; e < k * k; e += 32) {
        const int r = e / k, j = e % k;
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc = fma((double)Qf[r * ldk + i], Wm[i * ldk + j], acc);
        Z[r * ldk + j] = 1.5 * (double)Qf[r * ldk + j] - 0.5 * acc;
    }
    __syncwarp();
    // Wm = T Z (T tridiagonal: alpha on the diagonal, beta_r between r and r + 1)
    for (int e = lane; e < k * k; e += 32) {
        const int r = e / k, j = e % k;
        double acc = al[r] * Z[r * ldk + j];
        if (r > 0) acc = fma(be[r - 1], Z[(r - 1) * ldk + j], acc);
        if (r + 1 < k) acc = fma(be[r], Z[(r + 1) * ldk + j], acc);
        Wm[r * ldk + j] = acc;
    }
    __syncwarp();
    for (int i = lane; i < k; i += 32) {   // d_i = B_ii = z_i . (T z_i)
        double acc = 0.0;
        for (int r = 0; r < k; ++r) acc = fma(Z[r * ldk + i], Wm[r * ldk + i], acc);
        sv[i] = sqrt(fmax(acc, 0.0));
    }
    __syncwarp();
    for (int i = lane; i < k; i += 32) {   // h_i = sqrt(d_i) g_i + sum_j E_ij g_j / (sqrt(d_i) + sqrt(d_j))
        double h = sv[i] * Z[i];            // g_j = Z[0][j]
        for (int j = 0; j < k; ++j) {
            if (j == i) continue;
            const double den = sv[i] + sv[j];
            if (!(den > 0.0)) continue;
            double eij = 0.0;
            for (int r = 0; r < k; ++r) eij = fma(Z[r * ldk + i], Wm[r * ldk + j], eij);
            h = fma(eij * Z[j], 1.0 / den, h);
        }
        hv[i] = h;
    }
    __syncwarp();
    for (int r = lane; r < k; r += 32) {
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc = fma(Z[r * ldk + i], hv[i], acc);
        out[r] = wn * acc;
    }
    __syncwarp();
    return true;
}

// ||c_k - [c_{k-1}; 0]|| / ||c_k||, summed in the same order on every lane
__device__ inline double lz_change(const double* ck, const double* cprev, int k) {
    double num = 0.0, den = 0.0;
    for (int r = 0; r < k; ++r) {
        const double old = r < k - 1 ? cprev[r] : 0.0;
        num += (ck[r] - old) * (ck[r] - old);
        den += ck[r] * ck[r];
    }
    return den > 0.0 ? sqrt(num / den) : 0.0;
}

// The stopping index is the smallest k >= 2 with ||c_k - c_{k-1}|| / ||c_k|| < tol
// whatever the check schedule: when the first check of a run (index firstk + 1) already
// passes, earlier indices are examined backwards.  lastk[s] is the last index whose c was
// formed (-1 at the start of a run), lastk[S + s] the first one.  Launched with 32 threads
// and lz_tridiag_smem(kmax) bytes of dynamic shared memory; every lane
// follows the same control flow and lane 0 alone writes the per-suspension scalars.
__global__ void __launch_bounds__(32) k_lz_tridiag(int S, int j, const int* __restrict__ jdev, const double* __restrict__ h, int cols,
                                                   const double* __restrict__ wn2, double* __restrict__ alpha,
                                                   double* __restrict__ betav, const double* __restrict__ Wnorm,
                                                   double* __restrict__ cvec, double* __restrict__ err,
                                                   int* __restrict__ active, int* __restrict__ kcount,
                                                   int* __restrict__ lastk, double* __restrict__ scal, double tol,
                                                   const int* __restrict__ fixed, int* __restrict__ hint, int kmax,
                                                   const long long* __restrict__ susp_blob_off, int* __restrict__ status,
                                                   double* __restrict__ qbuf) {
    extern __shared__ __align__(16) unsigned char lz_smem[];
    const int s = blockIdx.x;
    const int lane = threadIdx.x;
    const bool lead = lane == 0;
    if (!active[s]) {
        if (lead) scal[s] = 0.0;
        return;
    }
    if (jdev) j = *jdev;
    const int k = j + 1;
    double beta = sqrt(fmax(wn2[(long long)s * cols], 0.0));
    double* al = alpha + (long long)s * kmax;
    double* be = betav + (long long)s * kmax;
    const double aj = h[(long long)s * cols + j];
    const double a0 = j == 0 ? aj : al[0];
    // Krylov space exhausted (k reached the dimension) or numerically invariant: exact stop
    const long long dim = 3 * (susp_blob_off[s + 1] - susp_blob_off[s]);
    if (k >= dim || beta <= 1e-14 * fmax(fabs(a0), fabs(aj))) beta = 0.0;
    if (lead) {
        al[j] = aj;
        be[j] = beta;
        scal[s] = beta > 0.0 ? 1.0 / beta : 0.0;
        kcount[s] = k;
    }
    __syncwarp();   // al[j], be[j] visible to every lane
    const bool fixed_mode = fixed != nullptr && fixed[s] > 0;
    // checks start a little before this suspension's previous count (hint[s]; 0 = none)
    const int hs = fixed_mode ? 0 : hint[s];
    const int kstart = hs > 0 ? max(2, hs - max(4, hs / 16)) : 2;
    const bool compute = fixed_mode ? (k >= fixed[s] || k >= kmax || beta == 0.0)
                                    : (k >= kstart || k >= kmax || beta == 0.0);
    if (!compute) return;
    double* cs_ = cvec + (long long)s * kmax;   // c of the last formed index
    const double wn = Wnorm[s];
    double* cur = reinterpret_cast<double*>(lz_smem);
    double* ck = cur + kmax;
    double* cm = ck + kmax;
    double* best = cm + kmax;
    double* Q = qbuf ? qbuf + (long long)s * lz_q_doubles_dev(kmax) : best + kmax;
    const int ldq = lz_ldq(kmax);
    const bool check32 = !fixed_mode && tol >= 1e-5;   // FP32 stopping test, FP64 result
    if (!lz_sqrt_e1(al, be, k, wn, Q, ldq, cur, check32)) {
        if (lead) {
            atomicExch(status, 2);
            active[s] = 0;
            err[s] = 1.0;
        }
        return;
    }
    if (fixed_mode) {
        for (int r = lane; r < k; r += 32) cs_[r] = cur[r];
        if (lead) {
            err[s] = 0.0;
            active[s] = 0;
        }
        return;
    }
    const int prevk = lastk[s], firstk = lastk[S + s];
    double ee = beta == 0.0 ? 0.0 : 1.0;
    bool stop = beta == 0.0;
    int kstar = k;
    if (prevk == k - 1) {
        ee = lz_change(cur, cs_, k);
        if (ee < tol) {
            stop = true;
            if (firstk == k - 1) {   // no check was possible at k - 1: look further back
                for (int r = lane; r < k; r += 32) {
                    best[r] = cur[r];
                    if (r < k - 1) ck[r] = cs_[r];
                }
                __syncwarp();
                double best_err = ee;
                for (int kk = k - 1; kk >= 2; --kk) {
                    if (!lz_sqrt_e1(al, be, kk - 1, wn, Q, ldq, cm, check32)) break;
                    const double e2 = lz_change(ck, cm, kk);
                    if (!(e2 < tol)) break;
                    kstar = kk;
                    best_err = e2;
                    __syncwarp();   // every lane has read ck and cm
                    for (int r = lane; r < kk; r += 32) {
                        best[r] = ck[r];
                        if (r < kk - 1) ck[r] = cm[r];
                    }
                    __syncwarp();
                }
                __syncwarp();
                for (int r = lane; r < kstar; r += 32) cur[r] = best[r];
                __syncwarp();
                ee = best_err;
            }
        }
    }
    if (k >= kmax) stop = true;
    if (stop && check32) {   // the result at the stopping index, in FP64
        __syncwarp();
        const bool ok = kstar <= GDC_LZ_REFINE_MAX ? lz_sqrt_e1_refined(al, be, kstar, wn, Q, cur)
                                                   : lz_sqrt_e1(al, be, kstar, wn, Q, ldq, cur, false);
        if (!ok) {
            if (lead) {
                atomicExch(status, 2);
                active[s] = 0;
                err[s] = 1.0;
            }
            return;
        }
    }
    __syncwarp();   // every lane has read lastk and cs_ before they are written
    for (int r = lane; r < kstar; r += 32) cs_[r] = cur[r];
    if (lead) {
        if (firstk < 0) lastk[S + s] = k;
        lastk[s] = k;
        kcount[s] = kstar;
        err[s] = ee;
        if (stop) {
            active[s] = 0;
            hint[s] = kstar;
        }
    }
}
__global__ void k_lz_reset(int S, int* __restrict__ lastk) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) {
        lastk[s] = -1;
        lastk[S + s] = -1;
    }
}

void krylov_init_attributes() {
    cudaFuncSetAttribute(k_lz_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)lz_tridiag_smem(GDC_MAX_LANCZOS));
}

gdc_status lanczos_sqrt(gdc_ctx* c, const double* W, double* out, double scale, int fixed_mode,
                        int* iters_out, double* err_out) {
    const int prec = c->p.precision;
    const long long n = 3LL * c->NBL;
    const gdc::Seg& sg = c->seg_lz;
    const int cols = c->red_cols;
    const int kmax = c->kmax;
    gdc_status st = GDC_OK;
    // convergence checks start a little before the previous run's count
    seg_mdot(c, sg, W, 0, 1, W, c->lz_h, cols);
    ++c->n_launch, k_lz_start<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, c->lz_h, cols, c->lz_Wnorm, c->lz_scal,
                                                                          c->lz_active, c->lz_k, c->lz_err);
    ++c->n_launch, k_lz_reset<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, c->lz_lastk);
    ++c->n_launch, k_seg_scale<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, W, c->lz_scal, c->lz_V);
    std::vector<int> act(c->S);
    for (int j = 0; j < kmax; ++j) {
        const double* Vj = c->lz_V + (long long)j * n;
        c->mv_active = c->lz_active;   // suspensions that have stopped need no product
        lz_operator(c, prec, Vj, c->lz_w);
        c->mv_active = nullptr;
        // w = M v_j orthogonalised against v_0..v_j twice (full reorthogonalisation)
        seg_mdot(c, sg, c->lz_V, n, j + 1, c->lz_w, c->lz_h, cols);
        ++c->n_launch, k_mupdate<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->lz_V, n, j + 1, nullptr, c->lz_h, cols, c->lz_w);
        seg_mdot(c, sg, c->lz_V, n, j + 1, c->lz_w, c->gm_h2, cols);
        ++c->n_launch, k_mupdate<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->lz_V, n, j + 1, nullptr, c->gm_h2, cols, c->lz_w);
        ++c->n_launch, k_add_cols<<<c->S, 128, 0, c->stream>>>(j + 1, nullptr, c->lz_h, c->gm_h2, cols);
        seg_mdot(c, sg, c->lz_w, 0, 1, c->lz_w, c->gm_h2, cols);
        ++c->n_launch, k_lz_tridiag<<<c->S, 32, lz_launch_smem(c), c->stream>>>(
            c->S, j, nullptr, c->lz_h, cols, c->gm_h2, c->lz_alpha, c->lz_beta, c->lz_Wnorm, c->lz_c, c->lz_err, c->lz_active,
            c->lz_k, c->lz_lastk, c->lz_scal, c->p.lanczos_tol, fixed_mode ? c->lz_fix : nullptr, c->lz_hint, kmax, c->susp_blob_off,
            c->dev_status, c->lz_qbuf_on ? c->lz_qbuf : nullptr);
        ++c->n_launch, k_seg_scale<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->lz_w, c->lz_scal,
                                                                       c->lz_V + (long long)(j + 1) * n);
        if ((st = sync_read(c, c->lz_active, act.data(), sizeof(int) * c->S)) != GDC_OK) return st;
        bool still = false;
        for (int s = 0; s < c->S; ++s) still = still || act[s];
        if (!still) break;
    }
    lz_result(c, scale, out);
    std::vector<int> ks(c->S);
    std::vector<double> errs(c->S);
    if ((st = sync_read(c, c->lz_k, ks.data(), sizeof(int) * c->S)) != GDC_OK) return st;
    if ((st = sync_read(c, c->lz_err, errs.data(), sizeof(double) * c->S)) != GDC_OK) return st;
    int kk = 0;
    double ee = 0.0;
    for (int s = 0; s < c->S; ++s) {
        kk = std::max(kk, ks[s]);
        ee = std::max(ee, errs[s]);
    }
    if (iters_out) *iters_out = kk;
    if (err_out) *err_out = ee;
    if (!fixed_mode && ee > c->p.lanczos_tol && kk >= kmax)
        return fail(c, GDC_ERR_NOT_CONVERGED, "Lanczos reached lanczos_max_iter");
    return cuda_check(c, cudaGetLastError(), "Lanczos launch");
}

// ---- graph mode: the Krylov loops as CUDA-graph WHILE nodes ---------------------------
//
// The loops above decide convergence on the host, one small device-to-host read per
// iteration.  In graph mode the same kernels run with their iteration index read from
// device memory (LoopCtl) and the last kernel of every iteration sets the condition of the
// WHILE node, so a whole step runs without a host round trip.  The arithmetic, and hence
// every result, is the same as in the host-driven loops.

// OR of flag[0..S) on one warp
__device__ inline int warp_any_flag(int S, const int* __restrict__ flag) {
    int any = 0;
    for (int s = threadIdx.x; s < S; s += 32) any |= flag[s] != 0;
    return __any_sync(0xffffffffu, any);
}

__global__ void __launch_bounds__(32) k_lz_begin(int S, const int* __restrict__ active, LoopCtl* ctl, int kmax,
                                                 cudaGraphConditionalHandle h) {
    const int any = warp_any_flag(S, active);
    if (threadIdx.x == 0) {
        ctl->lz_j = 0;
        cudaGraphSetConditional(h, (any && kmax > 0) ? 1u : 0u);
    }
}

__global__ void __launch_bounds__(32) k_lz_next(int S, const int* __restrict__ active, LoopCtl* ctl, int kmax,
                                                cudaGraphConditionalHandle h) {
    const int any = warp_any_flag(S, active);
    if (threadIdx.x == 0) {
        const int j = ++ctl->lz_j;
        cudaGraphSetConditional(h, (any && j < kmax) ? 1u : 0u);
    }
}

// the host-side summary of the eager loop, on the device: largest count and change
__global__ void __launch_bounds__(32) k_lz_finish(int S, const int* __restrict__ kcount, const double* __restrict__ err,
                                                  int fixed_mode, double tol, int kmax, const LoopCtl* ctl,
                                                  StepReport* rep, int run) {
    int kk = 0;
    double ee = 0.0;
    for (int s = threadIdx.x; s < S; s += 32) {
        kk = max(kk, kcount[s]);
        ee = fmax(ee, err[s]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kk = max(kk, __shfl_xor_sync(0xffffffffu, kk, o));
        ee = fmax(ee, __shfl_xor_sync(0xffffffffu, ee, o));
    }
    if (threadIdx.x == 0) {
        rep->lz_iters[run] = kk;
        rep->lz_err[run] = ee;
        rep->lz_notconv[run] = (!fixed_mode && ee > tol && kk >= kmax) ? 1 : 0;
        rep->lz_exec[run] = ctl->lz_j;
    }
}

__global__ void k_gm_reset(LoopCtl* ctl) {
    ctl->gm_j = 0;
    ctl->gm_total = 0;
    ctl->gm_checks = 0;
    ctl->gm_outer = 0;
}

// after k_gm_start: the residual check of a cycle boundary, and the outer loop's condition
__global__ void __launch_bounds__(32) k_gm_check(int S, const int* __restrict__ outer, const double* __restrict__ res,
                                                 LoopCtl* ctl, int max_iter, StepReport* rep,
                                                 cudaGraphConditionalHandle h, cudaGraphConditionalHandle hacc,
                                                 int mixed) {
    int any = 0, bad = 0;
    double rmax = 0.0;
    for (int s = threadIdx.x; s < S; s += 32) {
        const double r = res[s];
        any |= outer[s] != 0;
        bad |= !isfinite(r);
        rmax = fmax(rmax, r);
    }
    any = __any_sync(0xffffffffu, any);
    bad = __any_sync(0xffffffffu, bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if (threadIdx.x != 0) return;
    rep->gm_residual = rmax;
    rep->gm_cycles = ctl->gm_checks++;
    int go = 0;
    if (bad)
        rep->gm_bad = 1;
    else if (!any)
        rep->gm_converged = 1;
    else if (ctl->gm_total >= max_iter)
        rep->gm_notconv = 1;
    else
        go = 1;
    ctl->gm_j = 0;
    cudaGraphSetConditional(h, go ? 1u : 0u);
    // the next residual: recomputed accurately, or (mixed precision, small residuals) updated
    cudaGraphSetConditional(hacc, (!mixed || !(rmax <= GDC_RESID_UPDATE)) ? 1u : 0u);
}

__global__ void k_count(int* counter) { ++*counter; }

__global__ void k_gm_inner_begin(LoopCtl* ctl, cudaGraphConditionalHandle h) {
    ctl->gm_outer++;
    cudaGraphSetConditional(h, 1u);
}

__global__ void __launch_bounds__(32) k_gm_inner_next(int S, const int* __restrict__ active, LoopCtl* ctl,
                                                      int max_iter, cudaGraphConditionalHandle h) {
    const int any = warp_any_flag(S, active);
    if (threadIdx.x == 0) {
        ctl->gm_j++;
        const int total = ++ctl->gm_total;
        cudaGraphSetConditional(h, (any && total < max_iter) ? 1u : 0u);
    }
}

__global__ void k_gm_finish(const LoopCtl* ctl, StepReport* rep) {
    rep->gm_total = ctl->gm_total;
    rep->gm_outer = ctl->gm_outer;
}

// ---- capture helpers -------------------------------------------------------------

static void cap_chk(gdc_ctx* c, cudaError_t e) {
    if (e != cudaSuccess && c->cap_err == cudaSuccess) c->cap_err = e;
}

// a condition handle of the graph the library's stream is capturing into
cudaGraphConditionalHandle cap_cond(gdc_ctx* c) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    cap_chk(c, cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle h = 0;
    if (g) cap_chk(c, cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    return h;
}

// Appends a WHILE node on h after the work captured so far and redirects the library's
// stream into the node's body graph (a capture stream of its own, one per nesting level).
void cap_while_begin(gdc_ctx* c, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    cap_chk(c, cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, &edges, &nd));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    cap_chk(c, cudaGraphAddNode(&node, g, deps, edges, nd, &np));
    cap_chk(c, cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    const int d = ++c->cap_depth;
    c->cap_saved[d] = c->stream;
    if (d >= 3 || c->cap_err != cudaSuccess) {
        cap_chk(c, cudaErrorNotSupported);
        return;
    }
    cap_chk(c, cudaStreamBeginCaptureToGraph(c->cap_stream[d], np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed));
    c->stream = c->cap_stream[d];
}

// Ends the body capture; the kernels launched since launches_before run once per
// iteration, which the report slot counts.
void cap_while_end(gdc_ctx* c, int report_slot, unsigned long long launches_before) {
    const int d = c->cap_depth;
    if (d < 3 && c->stream == c->cap_stream[d]) {
        cudaGraph_t out = nullptr;
        cap_chk(c, cudaStreamEndCapture(c->stream, &out));
    }
    c->stream = c->cap_saved[d];
    c->cap_depth = d - 1;
    c->graph_loops.push_back({report_slot, c->n_launch - launches_before});
    c->n_launch = launches_before;
}

// Appends an IF/ELSE node on h and redirects the library's stream into its first body
// (run when the condition is non-zero); cap_ifelse_next switches to the second body,
// cap_ifelse_end returns to the enclosing graph.  Each body's kernels run once per
// execution of that branch, which the report slot counts.
void cap_ifelse_begin(gdc_ctx* c, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    cap_chk(c, cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, &edges, &nd));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 2;
    cudaGraphNode_t node = nullptr;
    cap_chk(c, cudaGraphAddNode(&node, g, deps, edges, nd, &np));
    cap_chk(c, cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    const int d = ++c->cap_depth;
    c->cap_saved[d] = c->stream;
    if (d >= 3 || c->cap_err != cudaSuccess) {
        cap_chk(c, cudaErrorNotSupported);
        return;
    }
    c->cap_bodies[0] = np.conditional.phGraph_out[0];
    c->cap_bodies[1] = np.conditional.phGraph_out[1];
    cap_chk(c, cudaStreamBeginCaptureToGraph(c->cap_stream[d], c->cap_bodies[0], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed));
    c->stream = c->cap_stream[d];
}

void cap_ifelse_next(gdc_ctx* c, int report_slot, unsigned long long launches_before) {
    const int d = c->cap_depth;
    if (d < 3 && c->stream == c->cap_stream[d]) {
        cudaGraph_t out = nullptr;
        cap_chk(c, cudaStreamEndCapture(c->stream, &out));
        cap_chk(c, cudaStreamBeginCaptureToGraph(c->cap_stream[d], c->cap_bodies[1], nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeRelaxed));
    }
    c->graph_loops.push_back({report_slot, c->n_launch - launches_before});
    c->n_launch = launches_before;
}

void cap_ifelse_end(gdc_ctx* c, int report_slot, unsigned long long launches_before) {
    cap_while_end(c, report_slot, launches_before);
}

// ---- the loops -------------------------------------------------------------------

void lanczos_sqrt_graph(gdc_ctx* c, const double* W, double* out, double scale, int fixed_mode, int run) {
    const int prec = c->p.precision;
    const long long n = 3LL * c->NBL;
    const gdc::Seg& sg = c->seg_lz;
    const int cols = c->red_cols;
    const int kmax = c->kmax;
    int* jd = &c->ctl->lz_j;
    seg_mdot(c, sg, W, 0, 1, W, c->lz_h, cols);
    ++c->n_launch, k_lz_start<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, c->lz_h, cols, c->lz_Wnorm, c->lz_scal,
                                                                          c->lz_active, c->lz_k, c->lz_err);
    ++c->n_launch, k_lz_reset<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, c->lz_lastk);
    ++c->n_launch, k_seg_scale_slot<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, W, c->lz_scal, c->lz_V, n, nullptr,
                                                                        0, c->lz_vcur);
    const cudaGraphConditionalHandle h = cap_cond(c);
    ++c->n_launch, k_lz_begin<<<1, 32, 0, c->stream>>>(c->S, c->lz_active, c->ctl, kmax, h);
    cap_while_begin(c, h);
    const unsigned long long before = c->n_launch;
    c->mv_active = c->lz_active;
    lz_operator(c, prec, c->lz_vcur, c->lz_w);
    c->mv_active = nullptr;
    seg_mdot(c, sg, c->lz_V, n, 1, c->lz_w, c->lz_h, cols, jd, kmax);
    ++c->n_launch, k_mupdate<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->lz_V, n, 1, jd, c->lz_h, cols, c->lz_w);
    seg_mdot(c, sg, c->lz_V, n, 1, c->lz_w, c->gm_h2, cols, jd, kmax);
    ++c->n_launch, k_mupdate<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->lz_V, n, 1, jd, c->gm_h2, cols, c->lz_w);
    ++c->n_launch, k_add_cols<<<c->S, 128, 0, c->stream>>>(1, jd, c->lz_h, c->gm_h2, cols);
    seg_mdot(c, sg, c->lz_w, 0, 1, c->lz_w, c->gm_h2, cols);
    ++c->n_launch, k_lz_tridiag<<<c->S, 32, lz_launch_smem(c), c->stream>>>(
        c->S, 0, jd, c->lz_h, cols, c->gm_h2, c->lz_alpha, c->lz_beta, c->lz_Wnorm, c->lz_c, c->lz_err, c->lz_active,
        c->lz_k, c->lz_lastk, c->lz_scal, c->p.lanczos_tol, fixed_mode ? c->lz_fix : nullptr, c->lz_hint, kmax,
        c->susp_blob_off, c->dev_status, c->lz_qbuf_on ? c->lz_qbuf : nullptr);
    ++c->n_launch, k_seg_scale_slot<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->lz_w, c->lz_scal, c->lz_V, n, jd,
                                                                        1, c->lz_vcur);
    ++c->n_launch, k_lz_next<<<1, 32, 0, c->stream>>>(c->S, c->lz_active, c->ctl, kmax, h);
    cap_while_end(c, REP_LZ0 + run, before);
    lz_result(c, scale, out);
    ++c->n_launch, k_lz_finish<<<1, 32, 0, c->stream>>>(c->S, c->lz_k, c->lz_err, fixed_mode, c->p.lanczos_tol, kmax,
                                                        c->ctl, c->rep, run);
}

void gmres_solve_graph(gdc_ctx* c, const double* b, double* x) {
    const int prec = c->p.precision;
    const int m = c->m;
    const long long n = c->ngm;
    const gdc::Seg& sg = c->seg_gm;
    const int cols = c->red_cols;
    const double tol = c->p.gmres_tol;
    const double inner_tol = prec == GDC_FP32_MIXED ? 0.1 * tol : tol;
    const int max_iter = c->p.gmres_max_iter;
    int* jd = &c->ctl->gm_j;
    seg_mdot(c, sg, b, 0, 1, b, c->gm_h, cols);
    ++c->n_launch, k_sqrt_col0<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, c->gm_h, cols, c->gm_bnorm);
    cap_chk(c, cudaMemsetAsync(x, 0, sizeof(double) * n, c->stream));
    cap_chk(c, cudaMemcpyAsync(c->gm_r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    ++c->n_launch, k_gm_reset<<<1, 1, 0, c->stream>>>(c->ctl);
    // first residual check (r = b)
    seg_mdot(c, sg, c->gm_r, 0, 1, c->gm_r, c->gm_h2, cols);
    ++c->n_launch, k_gm_start<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, c->gm_h2, c->gm_bnorm, tol, cols,
                                                                          c->gm_res, c->gm_active, c->gm_g, c->gm_scal,
                                                                          m + 1, c->gm_j, c->gm_active + c->S);
    const cudaGraphConditionalHandle ho = cap_cond(c), hacc = cap_cond(c);
    const int mixed = prec == GDC_FP32_MIXED;
    ++c->n_launch, k_gm_check<<<1, 32, 0, c->stream>>>(c->S, c->gm_active + c->S, c->gm_res, c->ctl, max_iter, c->rep,
                                                       ho, hacc, mixed);
    cap_while_begin(c, ho);
    const unsigned long long before_o = c->n_launch;
    {
        // one restart / refinement cycle
        ++c->n_launch, k_seg_scale_slot<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_r, c->gm_scal, c->gm_V, n,
                                                                            nullptr, 0, c->gm_vcur);
        const cudaGraphConditionalHandle hi = cap_cond(c);
        ++c->n_launch, k_gm_inner_begin<<<1, 1, 0, c->stream>>>(c->ctl, hi);
        cap_while_begin(c, hi);
        const unsigned long long before_i = c->n_launch;
        {
            launch_precond(c, c->gm_vcur, c->gm_z, prec == GDC_FP32_MIXED);
            c->mv_active = c->gm_active;
            saddle_op(c, prec, c->gm_z, c->gm_w);
            c->mv_active = nullptr;
            seg_mdot(c, sg, c->gm_V, n, 1, c->gm_w, c->gm_h, cols, jd, m);
            ++c->n_launch, k_mupdate<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_V, n, 1, jd, c->gm_h, cols, c->gm_w);
            seg_mdot(c, sg, c->gm_V, n, 1, c->gm_w, c->gm_h2, cols, jd, m);
            ++c->n_launch, k_mupdate<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_V, n, 1, jd, c->gm_h2, cols, c->gm_w);
            ++c->n_launch, k_add_cols<<<c->S, 128, 0, c->stream>>>(1, jd, c->gm_h, c->gm_h2, cols);
            seg_mdot(c, sg, c->gm_w, 0, 1, c->gm_w, c->gm_h2, cols);
            ++c->n_launch, k_gm_arnoldi<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(
                c->S, 0, jd, m, c->gm_h, cols, c->gm_h2, c->gm_H, c->gm_cs, c->gm_sn, c->gm_g, c->gm_bnorm, inner_tol,
                c->gm_res + c->S, c->gm_active, c->gm_j, c->gm_scal);
            ++c->n_launch, k_seg_scale_slot<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_w, c->gm_scal, c->gm_V,
                                                                                n, jd, 1, c->gm_vcur);
            ++c->n_launch, k_gm_inner_next<<<1, 32, 0, c->stream>>>(c->S, c->gm_active, c->ctl, max_iter, hi);
        }
        cap_while_end(c, REP_GM_TOTAL, before_i);
        // x += P^-1 V y
        ++c->n_launch, k_gm_backsolve<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(c->S, m, c->gm_H, c->gm_g, c->gm_j,
                                                                                  c->gm_y, cols);
        ++c->n_launch, k_combine<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, c->gm_V, n, c->gm_j, c->gm_y, cols,
                                                                     nullptr, c->gm_w);
        launch_precond(c, c->gm_w, c->gm_z, prec == GDC_FP32_MIXED);   // the correction e of this cycle
        ++c->n_launch, k_axpy_chunks<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, 1.0, c->gm_z, x);
        // the residual: recomputed, r = b - A x (accurate product), or updated, r <- r - A e
        // (FP32 product of the small correction), as k_gm_check decided
        cap_ifelse_begin(c, hacc);
        {
            const unsigned long long before_a = c->n_launch;
            saddle_op(c, prec == GDC_FP32_MIXED ? GDC_PREC_DF64 : GDC_FP64, x, c->gm_w);
            ++c->n_launch, k_sub_chunks<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, b, c->gm_w, c->gm_r);
            ++c->n_launch, k_count<<<1, 1, 0, c->stream>>>(&c->rep->gm_df);
            cap_ifelse_next(c, REP_GM_DF, before_a);
            const unsigned long long before_u = c->n_launch;
            saddle_op(c, GDC_FP32_MIXED, c->gm_z, c->gm_w);
            ++c->n_launch, k_axpy_chunks<<<sg.n_chunks, 256, 0, c->stream>>>(sg.chunks, -1.0, c->gm_w, c->gm_r);
            cap_ifelse_end(c, REP_GM_UPD, before_u);
        }
        seg_mdot(c, sg, c->gm_r, 0, 1, c->gm_r, c->gm_h2, cols);
        ++c->n_launch, k_gm_start<<<ceil_div(c->S, 128), 128, 0, c->stream>>>(
            c->S, c->gm_h2, c->gm_bnorm, tol, cols, c->gm_res, c->gm_active, c->gm_g, c->gm_scal, m + 1, c->gm_j,
            c->gm_active + c->S);
        ++c->n_launch, k_gm_check<<<1, 32, 0, c->stream>>>(c->S, c->gm_active + c->S, c->gm_res, c->ctl, max_iter,
                                                           c->rep, ho, hacc, mixed);
    }
    cap_while_end(c, REP_GM_OUTER, before_o);
    ++c->n_launch, k_gm_finish<<<1, 1, 0, c->stream>>>(c->ctl, c->rep);
}

}  // namespace gdc
