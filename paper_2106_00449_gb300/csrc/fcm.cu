// Fluctuating force-coupling method (FCM) in a periodic cube: M_FCM = J L^-1 S and
// v-breve = J L^-1 D W (Sec. 4.2), discretised as Sec. 4.2 and Sec. 6.1 describe: Gaussian
// envelopes on an N^3 grid cut off beyond R_t, a Fourier spectral Stokes solve, trapezoidal
// averaging, and a fluctuating stress of six independent normals per grid point.
//
// GB300 layout: the grid work is bandwidth-bound, so it runs in FP32 on complex float2 grids
// of N^3 points, each holding two real fields as a + i b (their transforms are separated by
// conjugate symmetry in the solve): 0-1 the force density, 2-3 its velocity, 4-6 the six
// stress components, 7-8 the fluctuating velocity.  The last inverse pass (along x) writes a
// velocity packed per point (float4: x, y, z, 0) into one of two packed grids, deterministic
// and fluctuating; the fluctuating one is kept there for re-averaging.
//   * spreading is a gather: a block takes grid points of one binning cell (cells at least
//     R_t wide) and stages the blobs of the 27 cells around it that can reach them (blobs in
//     ascending index) in shared memory as FP32 offsets from the cell's corner; it is
//     deterministic and needs no atomics on the grid;
//   * the 3-D FFT is one launch per axis of self-sorting (Stockham) passes of radix 8 (then
//     4 or 2) with 8 points of a pencil per thread in registers, exchanged through shared
//     memory between passes (two exchanges for 512-point pencils); points are read once and
//     written once per axis, along x in the x pass and P consecutive x at a time in the y and
//     z passes;
//   * the solve (projection, 1/(eta k^2), the spectral divergence of the stress and the 1/N^3
//     of the inverse transform): for M_FCM lambda it runs between the forward and inverse z
//     passes in one launch (a block takes pencils with their mirrors, whose modes -k the split
//     of the two real fields needs), for v-breve it is one pass over the modes;
//   * averaging reads the packed velocity (one 16-byte load per point) and takes one warp per
//     blob; in each z-plane of the blob's box (at most 31 points per side) the rows that can
//     meet the sphere are one run of points, x fastest, dealt to the lanes in turn; each lane
//     sums its points of a plane in FP32 and the planes with FP32 compensation, and the lanes
//     are added in FP64 in a fixed order.
#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "philox.cuh"

struct gdc_fcm {
    gdc_fcm_params p{};
    cudaStream_t stream = 0;
    int N = 0, logN = 0;
    long long NG = 0;         // N^3
    double h = 0.0;           // grid spacing
    int nc = 2;               // binning cells per side
    float2* tw = nullptr;     // N/2 forward twiddles exp(-2 pi i j / N)
    float2* grid = nullptr;   // 9 complex grids
    float4* packed = nullptr; // 2 packed velocity grids: deterministic, fluctuating
    double4_32a* pw = nullptr;    // blob positions wrapped into the cube
    int* cell_of = nullptr;
    int* cnt = nullptr;
    int* start = nullptr;
    int* fill = nullptr;
    int* list = nullptr;
    float4* poff = nullptr;   // per list entry: the blob's offset from its cell's corner (FP32)
    float4* plam = nullptr;   // per list entry: its lambda (FP32)
    int* scan = nullptr;
    bool have_field = false;
    unsigned long long n_launch = 0;
    std::string err;
};

namespace gdc {

// pencils per FFT block: 2^LP (16 up to 256-point pencils, 8 for 512-point ones)

static int fcm_cells(const gdc_fcm_params& p) {
    return (int)std::min(128.0, std::max(2.0, std::floor(p.L / p.R_t)));
}

static const char* fcm_validate(const gdc_fcm_params* p) {
    if (!p) return "NULL params";
    if (p->N < 16 || p->N > 512 || (p->N & (p->N - 1))) return "N must be a power of two in [16, 512]";
    if (!(p->L > 0.0) || !std::isfinite(p->L)) return "L must be > 0";
    if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return "sigma must be > 0";
    if (!(p->R_t > 0.0) || !(p->R_t < 0.5 * p->L)) return "R_t must be in (0, L/2)";
    if (std::ceil(p->R_t / (p->L / p->N)) > 15.0) return "R_t must span at most 15 grid spacings";
    if (!(p->eta > 0.0) || !std::isfinite(p->eta)) return "eta must be > 0";
    if (p->max_blobs < 1) return "max_blobs must be >= 1";
    return nullptr;
}

// Sequential 256-byte aligned carving (base = nullptr only measures).
struct FcmCarver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(long long count) {
        off = (off + 255) / 256 * 256;
        T* q = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += sizeof(T) * (size_t)std::max(1LL, count);
        return q;
    }
};

static size_t fcm_carve(gdc_fcm* f, void* base) {
    FcmCarver w{static_cast<char*>(base)};
    const long long nc3 = (long long)f->nc * f->nc * f->nc;
    f->tw = w.take<float2>(f->N / 2);
    f->grid = w.take<float2>(9 * f->NG);
    f->packed = w.take<float4>(2 * f->NG);
    f->pw = w.take<double4_32a>(f->p.max_blobs);
    f->cell_of = w.take<int>(f->p.max_blobs);
    f->cnt = w.take<int>(nc3);
    f->start = w.take<int>(nc3);
    f->fill = w.take<int>(nc3);
    f->list = w.take<int>(f->p.max_blobs);
    f->poff = w.take<float4>(f->p.max_blobs);
    f->plam = w.take<float4>(f->p.max_blobs);
    f->scan = w.take<int>(scan_scratch(nc3));
    return w.off + 256;
}

static void fcm_layout(gdc_fcm* f, const gdc_fcm_params& p) {
    f->p = p;
    f->N = p.N;
    f->logN = 0;
    while ((1 << f->logN) < p.N) ++f->logN;
    f->NG = (long long)p.N * p.N * p.N;
    f->h = p.L / p.N;
    f->nc = fcm_cells(p);
}

// FFT blocks: TH threads (256; 512 or 1024 in the strided passes of 256- and 512-point
// pencils), each holding 8 points of one pencil, so a block transforms P = 8 TH / N pencils.
// Between passes the points go through shared memory, one row of fft_stride(N, P) float2 per
// pencil, point t of a row at fft_swz(t) = t ^ ((t >> 3) & 15) (a bijection of [0, N)): with
// these strides the 16 float2 of every half-warp (stride-8 writes of the first pass, grouped
// writes of the second, unit-stride reads) fall in distinct bank pairs for N >= 128,
// whichever way the threads map to pencils.
__host__ __device__ constexpr int fft_stride(int N, int P) {
    return N >= 128 ? N + (P >= 16 ? 1 : 16 / P) : (N == 32 ? 35 : N + 1);
}
__device__ __forceinline__ int fft_swz(int t) { return t ^ ((t >> 3) & 15); }
static size_t fft_smem(int N, int TH) {
    const int P = 8 * TH / N;
    return (size_t)(P * fft_stride(N, P) + N) * sizeof(float2);
}
// two rows per pencil (k_fft_x_pack, k_fcm_zsolve) and the twiddle table
static size_t fft_smem2(int N, int TH) {
    const int P = 8 * TH / N;
    return (size_t)(2 * P * fft_stride(N, P) + N) * sizeof(float2);
}
// Threads per block of the y and z passes for 256- and 512-point pencils (P consecutive x
// per warp row: 4 x 8 bytes = 32-byte runs at 256 threads and N = 512, 64 at 512, 128 at
// 1024).  Measured at 512^3 (M_FCM lambda / v-breve): 256 and 256 threads 16.6 / 15.6 ms,
// 512 and 512 15.0 / 13.6, 1024 and 1024 15.1 / 13.7, 256 and 1024 14.8 / 13.4, 512 and
// 1024 14.8 / 13.3: the z pass, whose points are N^2 apart, wants the longest runs.
#ifndef GDC_FFT_TH_Y
#define GDC_FFT_TH_Y 512
#endif
#ifndef GDC_FFT_TH_Z
#define GDC_FFT_TH_Z 1024
#endif
static int fft_threads(int N, int axis) { return N < 256 || axis == 0 ? 256 : (axis == 1 ? GDC_FFT_TH_Y : GDC_FFT_TH_Z); }

// ---- binning ------------------------------------------------------------------------

// Wraps each blob into the cube and bins it.
__global__ void k_fcm_bin(int n, const double* __restrict__ r, double L, int nc, double4_32a* __restrict__ pw,
                          int* __restrict__ cell_of, int* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double w = L / nc;
    double x[3];
    int c[3];
    for (int d = 0; d < 3; ++d) {
        double v = r[3LL * i + d];
        v -= L * floor(v / L);
        if (!(v < L) || !(v >= 0.0)) v = 0.0;   // v == L after rounding, or not finite
        c[d] = (int)fmin(fmax(floor(v / w), 0.0), nc - 1.0);
        x[d] = v;
    }
    pw[i] = make_double4_32a(x[0], x[1], x[2], 0.0);
    const int id = c[0] + nc * (c[1] + nc * c[2]);
    cell_of[i] = id;
    atomicAdd(cnt + id, 1);
}

__global__ void k_fcm_scatter(int n, const int* __restrict__ cell_of, const int* __restrict__ start,
                              int* __restrict__ fill, int* __restrict__ list) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int id = cell_of[i];
    list[start[id] + atomicAdd(fill + id, 1)] = i;
}

// ---- spreading (gather) -----------------------------------------------------------------

// Per entry e of the cell-sorted blob list: the blob's offset from the corner of its own cell
// (formed in FP64, rounded to FP32: a magnitude below the cell width) and its lambda in FP32,
// so that spreading stages blobs without FP64 arithmetic.
__global__ void k_fcm_stage_blobs(int n, double w, int nc, const int* __restrict__ list,
                                  const int* __restrict__ cell_of, const double4_32a* __restrict__ pw,
                                  const double* __restrict__ lam, float4* __restrict__ poff,
                                  float4* __restrict__ plam) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int j = list[e], id = cell_of[j];
    const int cx = id % nc, cy = (id / nc) % nc, cz = id / (nc * nc);
    const double4_32a p = pw[j];
    poff[e] = make_float4((float)(p.x - cx * w), (float)(p.y - cy * w), (float)(p.z - cz * w), 0.f);
    plam[e] = make_float4((float)lam[3LL * j], (float)lam[3LL * j + 1], (float)lam[3LL * j + 2], 0.f);
}

constexpr int SP_CHUNK = 128;    // blob entries examined per round (one per thread)

// f(x_g) = sum of lambda_j Delta_j(x_g).  One block per binning cell (cells at least R_t wide)
// and chunk of 128 PT of its grid points (blockIdx.y): the cell's grid points are those with
// floor(i nc / N) equal to its index on every axis (an exact integer partition of the grid),
// and every blob that can reach them lies in the 27 cells around it.  Those blobs are taken in
// a fixed order (cells in a fixed order, blobs in ascending index; rounds of SP_CHUNK) as FP32
// offsets from the cell's corner, nearest image to the cell's centre; a blob farther than R_t
// from the bounding box of the block's grid points is dropped (with at least 4 cells per side),
// the others are staged in shared memory in the same order (a ballot scan), and each thread
// sums them for its grid points with the minimum image in FP32.  A dropped blob misses every
// point of the block, so the sums are those of the full list, term for term.  Deterministic, no atomics on the grid.  With at least 4 cells per side every
// staged offset is within 2 cell widths of the cell, less than L/2 from any of its grid
// points, so the per-pair minimum image is the identity and WRAP = false drops it.  The image
// of a staged blob is chosen with a multiplication by 1/L (an FP64 division per coordinate
// there would make the FP64 pipe, 1/64 of the FP32 rate on this GPU, the kernel's limit).
template <int PT, bool WRAP>   // PT: grid points a thread keeps per round
__global__ void __launch_bounds__(128) k_fcm_spread(int N, double h, double L, double invL, double w, int nc,
                                                    const double4_32a* __restrict__ pw,
                                                    const int* __restrict__ cnt, const int* __restrict__ start,
                                                    const int* __restrict__ list, const double* __restrict__ lam,
                                                    const float4* __restrict__ poff, const float4* __restrict__ plam,
                                                    float R2, float l2s, float norm, float2* __restrict__ f,
                                                    long long NG) {
    __shared__ float4 sp[SP_CHUNK];
    __shared__ float4 sl[SP_CHUNK];
    __shared__ int wkept[SP_CHUNK / 32];
    __shared__ int c_start[27], c_off[28];
    __shared__ float base_off[3];   // offset of the cell's first grid point from its corner
    __shared__ double corner[3];    // the cell's corner (w = L / nc, the cell width)
    const int b = blockIdx.x;
    const int c3[3] = {b % nc, (b / nc) % nc, b / (nc * nc)};
    int g0[3], gn[3];
    for (int d = 0; d < 3; ++d) {
        g0[d] = (c3[d] * N + nc - 1) / nc;                  // first i with floor(i nc / N) = c
        gn[d] = ((c3[d] + 1) * N + nc - 1) / nc - g0[d];
    }
    const int npts = gn[0] * gn[1] * gn[2];
    if (npts <= (int)blockIdx.y * PT * 128) return;   // whole block: no points in this chunk
    // the neighbour cells (each once when the grid has fewer than 3 cells per side)
    const int no = nc >= 3 ? 3 : nc, o0 = nc >= 3 ? -1 : 0, ncell = no * no * no;
    if (threadIdx.x < ncell) {
        const int k = threadIdx.x;
        const int ox = o0 + k % no, oy = o0 + (k / no) % no, oz = o0 + k / (no * no);
        const int id = (c3[0] + ox + nc) % nc + nc * ((c3[1] + oy + nc) % nc + nc * ((c3[2] + oz + nc) % nc));
        c_start[k] = start[id];
        c_off[k + 1] = cnt[id];
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // the block's FP64 geometry, once (the FP64 pipe is slow)
        c_off[0] = 0;
        for (int k = 0; k < ncell; ++k) c_off[k + 1] += c_off[k];
        for (int d = 0; d < 3; ++d) {
            corner[d] = c3[d] * w;
            base_off[d] = (float)(g0[d] * h - corner[d]);
        }
    }
    __syncthreads();
    const int total = c_off[ncell];
    const float Lf = (float)L, hL = 0.5f * Lf, hf = (float)h;
    const double mid = 0.5 * w;
    const float wf = (float)w;
    {
        const int p0 = blockIdx.y * PT * 128;   // this block's chunk of the cell's grid points
        float gx[PT], gy[PT], gz[PT], ax[PT], ay[PT], az[PT];
        long long gi[PT];
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const int pt = p0 + q * 128 + (int)threadIdx.x;
            ax[q] = ay[q] = az[q] = 0.f;
            gi[q] = -1;
            gx[q] = gy[q] = gz[q] = 0.f;
            if (pt < npts) {
                // in FP32 from the block's base: FP64 arithmetic per point would load the FP64
                // pipe (1/64 of the FP32 rate) more than the pair loop loads the FP32 one
                const int jx = pt % gn[0], jy = (pt / gn[0]) % gn[1], jz = pt / (gn[0] * gn[1]);
                gx[q] = fmaf((float)jx, hf, base_off[0]);
                gy[q] = fmaf((float)jy, hf, base_off[1]);
                gz[q] = fmaf((float)jz, hf, base_off[2]);
                gi[q] = (g0[0] + jx) + (long long)N * ((g0[1] + jy) + (long long)N * (g0[2] + jz));
            }
        }
        // the bounding box of this block's grid points (whole x and y rows of the cell, the z
        // layers of the chunk) in the frame of the cell's corner, and the squared reach beyond
        // it, widened by 1e-4 against rounding (dropping is only ever conservative)
        const int layer = gn[0] * gn[1];
        const int zlo = p0 / layer, zhi = (min(p0 + PT * 128, npts) - 1) / layer;
        const float bx0 = base_off[0], bx1 = fmaf((float)(gn[0] - 1), hf, base_off[0]);
        const float by0 = base_off[1], by1 = fmaf((float)(gn[1] - 1), hf, base_off[1]);
        const float bz0 = fmaf((float)zlo, hf, base_off[2]), bz1 = fmaf((float)zhi, hf, base_off[2]);
        const float reach2 = R2 * 1.0001f;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int s0 = 0; s0 < total; s0 += SP_CHUNK) {
            const int e = s0 + (int)threadIdx.x;
            bool keep = false;
            float4 vp = make_float4(0.f, 0.f, 0.f, 0.f), vl = vp;
            __syncthreads();   // the previous round's staged blobs are no longer read
            if (e < total) {
                int k = 0;   // the neighbour cell of entry e: c_off[k] <= e < c_off[k + 1]
                for (int step = 16; step > 0; step >>= 1)
                    if (k + step <= ncell - 1 && c_off[k + step] <= e) k += step;
                const int pos = c_start[k] + (e - c_off[k]);
                if (WRAP) {   // few cells per side: the image nearest the cell's centre, in FP64
                    const int j = list[pos];
                    const double4_32a p = pw[j];
                    double rx = p.x - corner[0], ry = p.y - corner[1], rz = p.z - corner[2];
                    rx -= L * rint((rx - mid) * invL);
                    ry -= L * rint((ry - mid) * invL);
                    rz -= L * rint((rz - mid) * invL);
                    vp = make_float4((float)rx, (float)ry, (float)rz, 0.f);
                    vl = make_float4((float)lam[3LL * j], (float)lam[3LL * j + 1], (float)lam[3LL * j + 2], 0.f);
                    keep = true;
                } else {      // the neighbour cell's corner is o w from this cell's (o in {-1, 0, 1}^3)
                    const float4 q = poff[pos];
                    const float ox = (float)(k % 3 - 1), oy = (float)((k / 3) % 3 - 1), oz = (float)(k / 9 - 1);
                    vp = make_float4(fmaf(ox, wf, q.x), fmaf(oy, wf, q.y), fmaf(oz, wf, q.z), 0.f);
                    vl = plam[pos];
                    const float ex = fmaxf(fmaxf(bx0 - vp.x, vp.x - bx1), 0.f);
                    const float ey = fmaxf(fmaxf(by0 - vp.y, vp.y - by1), 0.f);
                    const float ez = fmaxf(fmaxf(bz0 - vp.z, vp.z - bz1), 0.f);
                    keep = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= reach2;
                }
            }
            // staged in entry order: the kept entries of lower warps, then of lower lanes
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) wkept[wid] = __popc(bal);
            __syncthreads();
            int base = 0, take = 0;
#pragma unroll
            for (int w2 = 0; w2 < SP_CHUNK / 32; ++w2) {
                const int c = wkept[w2];
                base += w2 < wid ? c : 0;
                take += c;
            }
            if (keep) {
                const int at = base + __popc(bal & ((1u << lane) - 1u));
                sp[at] = vp;
                sl[at] = vl;
            }
            __syncthreads();
            for (int j = 0; j < take; ++j) {
                const float4 pj = sp[j], lj = sl[j];
#pragma unroll
                for (int q = 0; q < PT; ++q) {
                    float dx = gx[q] - pj.x, dy = gy[q] - pj.y, dz = gz[q] - pj.z;
                    if (WRAP) {
                        dx = dx > hL ? dx - Lf : (dx < -hL ? dx + Lf : dx);
                        dy = dy > hL ? dy - Lf : (dy < -hL ? dy + Lf : dy);
                        dz = dz > hL ? dz - Lf : (dz < -hL ? dz + Lf : dz);
                    }
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (d2 <= R2) {
                        const float wt = norm * exp2f(-d2 * l2s);   // exp(-d2 / 2s^2)
                        ax[q] = fmaf(lj.x, wt, ax[q]);
                        ay[q] = fmaf(lj.y, wt, ay[q]);
                        az[q] = fmaf(lj.z, wt, az[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < PT; ++q)
            if (gi[q] >= 0) {
                f[gi[q]] = make_float2(ax[q], ay[q]);      // two real fields in one complex grid
                f[NG + gi[q]] = make_float2(az[q], 0.f);
            }
    }
}

// ---- FFT: self-sorting (Stockham) passes of radix 8, then 4 or 2; one axis per launch ----
//
// INV = 0: X_k = sum_n x_n exp(-2 pi i k n / N); INV = 1: the same with +i, unscaled.
// blockIdx.y picks the component grid (NG points apart).  Thread i of a pencil holds the
// points i + m T (m = 0..7, T = N/8) in registers.  A pass of radix R that follows
// sub-transforms of length p treats 8/R virtual threads v = i + u T: with k = v mod p it
// multiplies its inputs v + j N/R (j < R) by w^(j k), w = exp(-+2 pi i / (p R)), takes their
// R-point DFT and writes output j to (v - k) R + k + j p, so the points end in natural order
// after the last pass (Stockham's self-sorting order, no bit reversal).  The first pass
// reads straight from global memory and the last writes straight back, both at i + m T
// (coalesced along x in the x pass; P consecutive x per warp row in the y and z passes);
// in between the block exchanges its points through shared memory.

// x w (INV: x conj(w)), w a forward twiddle exp(-2 pi i m / N)
template <int INV>
__device__ __forceinline__ float2 fft_twiddle(float2 x, float2 w) {
    if (INV) w.y = -w.y;
    return make_float2(x.x * w.x - x.y * w.y, x.x * w.y + x.y * w.x);
}

// z times exp(-+2 pi i / 4) = -+i
template <int INV>
__device__ __forceinline__ float2 fft_rot4(float2 z) {
    return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// In-place R-point DFT of z[0..R-1] (R = 2, 4, 8), outputs in natural order.
template <int R, int INV>
__device__ __forceinline__ void fft_dft(float2* z) {
    if (R == 2) {
        const float2 a = z[0], b = z[1];
        z[0] = c_add(a, b);
        z[1] = c_sub(a, b);
    } else if (R == 4) {
        const float2 t0 = c_add(z[0], z[2]), t1 = c_sub(z[0], z[2]);
        const float2 t2 = c_add(z[1], z[3]), t3 = fft_rot4<INV>(c_sub(z[1], z[3]));
        z[0] = c_add(t0, t2);
        z[2] = c_sub(t0, t2);
        z[1] = c_add(t1, t3);
        z[3] = c_sub(t1, t3);
    } else {
        // even and odd halves by 4-point DFTs, then the radix-2 step with exp(-+2 pi i j / 8)
        float2 e[4] = {z[0], z[2], z[4], z[6]}, o[4] = {z[1], z[3], z[5], z[7]};
        fft_dft<4, INV>(e);
        fft_dft<4, INV>(o);
        const float r = 0.70710678118654752f;   // 1/sqrt(2)
        o[1] = fft_twiddle<INV>(o[1], make_float2(r, -r));
        o[2] = fft_rot4<INV>(o[2]);
        o[3] = fft_twiddle<INV>(o[3], make_float2(-r, -r));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            z[j] = c_add(e[j], o[j]);
            z[j + 4] = c_sub(e[j], o[j]);
        }
    }
}

// One pass of radix R after sub-transforms of length PL; LAST leaves the outputs in x at
// i + m T, the others write them to the pencil's shared-memory row and read the next pass's
// inputs back.
template <int INV, int LOGN, int R, int PL, bool LAST>
__device__ __forceinline__ void fft_pass(float2 (&x)[8], float2* row, const float2* tw, int i) {
    constexpr int N = 1 << LOGN, T = N / 8, V = 8 / R;
    float2 y[8];
#pragma unroll
    for (int u = 0; u < V; ++u) {
        const int v = i + u * T, k = v & (PL - 1);
        float2 z[8];
#pragma unroll
        for (int j = 0; j < R; ++j) z[j] = x[u + j * V];
        if (PL > 1) {
#pragma unroll
            for (int j = 1; j < R; ++j) z[j] = fft_twiddle<INV>(z[j], tw[(j * k * (N / (PL * R))) & (N - 1)]);
        }
        fft_dft<R, INV>(z);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (LAST)
                y[u + j * V] = z[j];
            else
                row[fft_swz((v - k) * R + k + j * PL)] = z[j];
        }
    }
    if (LAST) {
#pragma unroll
        for (int m = 0; m < 8; ++m) x[m] = y[m];
    } else {
        __syncthreads();
#pragma unroll
        for (int m = 0; m < 8; ++m) x[m] = row[fft_swz(i + m * T)];
        __syncthreads();   // the row is rewritten by the next pass
    }
}

template <int INV, int LOGN, int PASS>
__device__ __forceinline__ void fft_passes(float2 (&x)[8], float2* row, const float2* tw, int i) {
    constexpr int NP8 = LOGN / 3, REM = LOGN % 3, NPASS = NP8 + (REM ? 1 : 0);
    if constexpr (PASS < NPASS) {
        constexpr int R = PASS < NP8 ? 8 : (REM == 1 ? 2 : 4);
        fft_pass<INV, LOGN, R, (1 << (3 * PASS)), PASS == NPASS - 1>(x, row, tw, i);
        fft_passes<INV, LOGN, PASS + 1>(x, row, tw, i);
    }
}

template <int INV, int LOGN, int TH>
__global__ void __launch_bounds__(TH) k_fft(float2* __restrict__ data, long long NG, const float2* __restrict__ tw_g,
                                              int axis) {
    constexpr int N = 1 << LOGN, T = N / 8, P = TH / T, S = fft_stride(N, P);
    extern __shared__ float2 sm[];
    float2* tw = sm + P * S;   // exp(-2 pi i m / N), m = 0..N-1
    for (int j = threadIdx.x; j < N / 2; j += TH) {
        const float2 w = tw_g[j];
        tw[j] = w;
        tw[j + N / 2] = make_float2(-w.x, -w.y);
    }
    // pencil pid = blockIdx.x P + q of the N^2 along the axis; in the x pass a pencil's T
    // threads are consecutive, in the y and z passes the P pencils (consecutive x) are
    int q, i;
    if (axis == 0) {
        q = threadIdx.x / T;
        i = threadIdx.x % T;
    } else {
        q = threadIdx.x % P;
        i = threadIdx.x / P;
    }
    const long long pid = (long long)blockIdx.x * P + q;
    long long o, st;
    if (axis == 0) {
        o = pid << LOGN;
        st = 1;
    } else if (axis == 1) {
        o = (pid & (N - 1)) + ((pid >> LOGN) << (2 * LOGN));
        st = N;
    } else {
        o = (pid & (N - 1)) + ((pid >> LOGN) << LOGN);
        st = (long long)N * N;
    }
    float2* g = data + blockIdx.y * NG + o;
    float2 x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = g[(long long)(i + m * T) * st];
    __syncthreads();   // twiddle table complete
    fft_passes<INV, LOGN, 0>(x, sm + q * S, tw, i);
#pragma unroll
    for (int m = 0; m < 8; ++m) g[(long long)(i + m * T) * st] = x[m];
}

// The last inverse pass of a velocity, along x, with its packing: a block transforms P pencils
// of both complex grids u (u_x + i u_y at g, u_z at NG + g), one after the other, and writes
// the three real parts per point as (x, y, z, 0), the layout averaging gathers (one 16-byte
// load per point).  Same pencils and threads as the x pass of k_fft; the first grid's result
// waits in a second shared-memory row per pencil while the second is transformed.
template <int LOGN>
__global__ void __launch_bounds__(256, 4) k_fft_x_pack(const float2* __restrict__ u, long long NG,
                                                    const float2* __restrict__ tw_g, float4* __restrict__ out) {
    constexpr int TH = 256, N = 1 << LOGN, T = N / 8, P = TH / T, S = fft_stride(N, P);
    extern __shared__ float2 sm[];
    float2* park = sm + P * S + (threadIdx.x / T) * S;
    float2* tw = sm + 2 * P * S;
    for (int j = threadIdx.x; j < N / 2; j += TH) {
        const float2 w = tw_g[j];
        tw[j] = w;
        tw[j + N / 2] = make_float2(-w.x, -w.y);
    }
    const int q = threadIdx.x / T, i = threadIdx.x % T;
    const long long o = ((long long)blockIdx.x * P + q) << LOGN;
    float2 x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = u[o + i + m * T];
    __syncthreads();   // twiddle table complete
    fft_passes<1, LOGN, 0>(x, sm + q * S, tw, i);
#pragma unroll
    for (int m = 0; m < 8; ++m) park[i + m * T] = x[m];   // read back by this thread only
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = u[NG + o + i + m * T];
    fft_passes<1, LOGN, 0>(x, sm + q * S, tw, i);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const float2 a = park[i + m * T];
        out[o + i + m * T] = make_float4(a.x, a.y, x[m].x, 0.f);
    }
}

// ---- Fourier-space solve ------------------------------------------------------------------

struct Mode {
    bool keep;
    float kx, ky, kz, k2;
};

// The mode of grid indices (ix, iy, iz): its wave vector and whether it is kept (k != 0, no
// Nyquist component).
__device__ __forceinline__ Mode fcm_mode3(int ix, int iy, int iz, int N, float kunit) {
    const int half = N / 2;
    Mode m;
    m.keep = (ix | iy | iz) != 0 && ix != half && iy != half && iz != half;
    m.kx = kunit * (float)(ix < half ? ix : ix - N);
    m.ky = kunit * (float)(iy < half ? iy : iy - N);
    m.kz = kunit * (float)(iz < half ? iz : iz - N);
    m.k2 = m.kx * m.kx + m.ky * m.ky + m.kz * m.kz;
    return m;
}

__device__ __forceinline__ Mode fcm_mode(long long g, int N, float kunit) {
    return fcm_mode3((int)(g % N), (int)((g / N) % N), (int)(g / ((long long)N * N)), N, kunit);
}

// u = (I - k k^T / k^2) f / (eta k^2) / N^3 for one mode (complex f components)
__device__ __forceinline__ void fcm_project(const Mode& m, float scale_eta, float2 fx, float2 fy, float2 fz,
                                            float2& ux, float2& uy, float2& uz) {
    const float inv = scale_eta / m.k2;
    const float kfr = (m.kx * fx.x + m.ky * fy.x + m.kz * fz.x) / m.k2;
    const float kfi = (m.kx * fx.y + m.ky * fy.y + m.kz * fz.y) / m.k2;
    ux = make_float2((fx.x - m.kx * kfr) * inv, (fx.y - m.kx * kfi) * inv);
    uy = make_float2((fy.x - m.ky * kfr) * inv, (fy.y - m.ky * kfi) * inv);
    uz = make_float2((fz.x - m.kz * kfr) * inv, (fz.y - m.kz * kfi) * inv);
}

// Index of the mode -k.
__device__ __forceinline__ long long fcm_mirror(long long g, int N) {
    const int m = N - 1;
    const int ix = (int)(g % N), iy = (int)((g / N) % N), iz = (int)(g / ((long long)N * N));
    return ((N - ix) & m) + (long long)N * (((N - iy) & m) + (long long)N * ((N - iz) & m));
}

// The transforms A, B of two real fields from Z = FFT(a + i b) at k and -k:
// A(k) = (Z(k) + conj Z(-k)) / 2, B(k) = (Z(k) - conj Z(-k)) / (2i).
__device__ __forceinline__ void fcm_split(float2 zk, float2 zm, float2& A, float2& B) {
    A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    B = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
}

// A + i B for two transforms of real fields: the inverse transform gives a + i b.
__device__ __forceinline__ float2 fcm_join(float2 A, float2 B) { return make_float2(A.x - B.y, A.y + B.x); }

// The z passes of both transforms with the solve between them, in one launch.  F holds
// FFT_xy(f_x + i f_y) and FFT_xy(f_z) (x and y passes done), U receives the velocity's two grids
// (u_x + i u_y, u_z) before their inverse x and y passes, scaled for the inverse.  Splitting
// FFT(f_x + i f_y) into its two real fields needs the mode -k beside k, so a block takes H
// pencils (x, y) of consecutive x from the rows y = 0 .. N/2 together with their mirror
// pencils (-x, -y): per pencil it transforms both force grids along z, keeps the first
// spectrum in shared memory in natural order (the partner pencil reads its mode -k_z there),
// solves, and transforms the two velocity grids back along z.  The grids are read and written
// once instead of three times (forward z pass, solve, inverse z pass).  In the rows y = 0 and
// y = N/2 the pencils x > N/2 are the mirrors of N - x and come with them; the four pencils
// with x, y in {0, N/2} are their own mirrors.
// blocks per SM the fused kernel is compiled for (512 threads at 2 blocks per SM measured
// 9.89 ms per M_FCM lambda at 512^3 against 9.51 with 1,024 threads at 1)
#ifndef GDC_ZSOLVE_MINB
#define GDC_ZSOLVE_MINB 1
#endif
template <int LOGN, int TH>
__global__ void __launch_bounds__(TH, GDC_ZSOLVE_MINB) k_fcm_zsolve(const float2* __restrict__ F, float2* __restrict__ U, long long NG,
                                                   const float2* __restrict__ tw_g, float kunit, float scale_eta) {
    constexpr int N = 1 << LOGN, T = N / 8, P = TH / T, H = P / 2, S = fft_stride(N, P);
    extern __shared__ float2 sm[];
    float2* zr = sm + P * S;   // per pencil: its spectrum of f_x + i f_y, later its parked u_z
    float2* tw = zr + P * S;   // exp(-2 pi i m / N), m = 0..N-1
    for (int j = threadIdx.x; j < N / 2; j += TH) {
        const float2 w = tw_g[j];
        tw[j] = w;
        tw[j + N / 2] = make_float2(-w.x, -w.y);
    }
    // pencil q of the block: slot q mod H (x consecutive), side 0 the slot's pencil, 1 its mirror
    const int q = threadIdx.x % P, i = threadIdx.x / P, side = q / H;
    const long long s = (long long)blockIdx.x * H + q % H;
    const int sx = (int)(s & (N - 1)), sy = (int)(s >> LOGN);
    const bool self = (sx == 0 || sx == N / 2) && (sy == 0 || sy == N / 2);
    const bool slot = sy <= N / 2 && ((sy > 0 && sy < N / 2) || sx <= N / 2);
    const bool run = slot && !(side == 1 && self);   // the mirror side of a self-mirrored pencil idles
    const int px = side ? (N - sx) & (N - 1) : sx, py = side ? (N - sy) & (N - 1) : sy;
    const int partner = self ? q : (side ? q - H : q + H);
    const long long o = px + ((long long)py << LOGN), st = (long long)N * N;
    float2* row = sm + q * S;
    float2* zq = zr + q * S;
    float2 x[8], z1[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = run ? F[o + (long long)(i + m * T) * st] : make_float2(0.f, 0.f);
    __syncthreads();   // twiddle table complete
    fft_passes<0, LOGN, 0>(x, row, tw, i);
#pragma unroll
    for (int m = 0; m < 8; ++m) zq[i + m * T] = x[m];
#pragma unroll
    for (int m = 0; m < 8; ++m) z1[m] = run ? F[NG + o + (long long)(i + m * T) * st] : make_float2(0.f, 0.f);
    fft_passes<0, LOGN, 0>(z1, row, tw, i);
    __syncthreads();   // every pencil's spectrum of f_x + i f_y in shared memory
    const float2* zp = zr + partner * S;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int kz = i + m * T;
        const Mode md = fcm_mode3(px, py, kz, N, kunit);
        float2 o0 = make_float2(0.f, 0.f), o1 = o0;
        if (md.keep) {
            float2 fx, fy, ux, uy, uz;
            fcm_split(zq[kz], zp[(N - kz) & (N - 1)], fx, fy);
            fcm_project(md, scale_eta, fx, fy, z1[m], ux, uy, uz);
            o0 = fcm_join(ux, uy);
            o1 = uz;
        }
        row[kz] = o0;   // the exchange row is free here: parked until the spectra are read
        z1[m] = o1;
    }
    __syncthreads();   // the spectra are no longer read
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        zq[i + m * T] = z1[m];   // parked while u_x + i u_y is transformed
        x[m] = row[i + m * T];
    }
    __syncthreads();   // the first inverse pass rewrites the row
    fft_passes<1, LOGN, 0>(x, row, tw, i);
    if (run) {
#pragma unroll
        for (int m = 0; m < 8; ++m) U[o + (long long)(i + m * T) * st] = x[m];
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) z1[m] = zq[i + m * T];
    fft_passes<1, LOGN, 0>(z1, row, tw, i);
    if (run) {
#pragma unroll
        for (int m = 0; m < 8; ++m) U[NG + o + (long long)(i + m * T) * st] = z1[m];
    }
}

// Threads per block of k_fcm_zsolve (its shared memory: fft_smem2, 132-135 KB at 1024
// threads: 16 pencils of 512 points or 32 of 256).
#ifndef GDC_ZSOLVE_TH
#define GDC_ZSOLVE_TH 1024
#endif
static int zsolve_threads(int N) { return N >= 256 ? GDC_ZSOLVE_TH : 256; }

__device__ __forceinline__ float2 cadd3(float a, float2 x, float b, float2 y, float c, float2 z) {
    return make_float2(a * x.x + b * y.x + c * z.x, a * x.y + b * y.y + c * z.y);
}

// Z: FFT(W_xx + i W_yy), FFT(W_zz + i W_xy), FFT(W_xz + i W_yz); u: the velocity's transforms
// (u_x + i u_y, u_z), scaled for the inverse.
__global__ void k_fcm_solve_stress(long long NG, int N, float kunit, float scale_eta, const float2* __restrict__ Z,
                                   float2* __restrict__ u) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= NG) return;
    const Mode m = fcm_mode(g, N, kunit);
    float2 o0 = make_float2(0.f, 0.f), o1 = o0;
    if (m.keep) {
        const long long gm = fcm_mirror(g, N);
        float2 xx, yy, zz, xy, xz, yz, ux, uy, uz;
        fcm_split(Z[g], Z[gm], xx, yy);
        fcm_split(Z[NG + g], Z[NG + gm], zz, xy);
        fcm_split(Z[2 * NG + g], Z[2 * NG + gm], xz, yz);
        // (D W)_a = i k_b W_ab
        const float2 dx = cadd3(m.kx, xx, m.ky, xy, m.kz, xz);
        const float2 dy = cadd3(m.kx, xy, m.ky, yy, m.kz, yz);
        const float2 dz = cadd3(m.kx, xz, m.ky, yz, m.kz, zz);
        fcm_project(m, scale_eta, make_float2(-dx.y, dx.x), make_float2(-dy.y, dy.x), make_float2(-dz.y, dz.x), ux, uy,
                    uz);
        o0 = fcm_join(ux, uy);
        o1 = uz;
    }
    u[g] = o0;
    u[NG + g] = o1;
}

// ---- fluctuating stress ---------------------------------------------------------------------

// Six normals per grid point (Box-Muller in FP32: the grid is FP32, and FP64 logarithms and
// sines for 6 N^3 draws would dominate the Brownian velocity on GB300).
__global__ void k_fcm_stress(long long NG, unsigned long long seed, unsigned owner, unsigned long long step, float sd,
                             float so, float2* __restrict__ W) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= NG) return;
    const uint2 key = make_uint2((unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
    float n[6];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const uint4 x = philox4x32_10(make_uint4((unsigned)(3 * g + q), owner, (unsigned)(step & 0xffffffffull), 2u), key);
        normals_f32(x, n[2 * q], n[2 * q + 1]);
    }
    // three complex grids, two real components each: xx + i yy, zz + i xy, xz + i yz
    W[g] = make_float2(sd * n[0], sd * n[1]);
    W[NG + g] = make_float2(sd * n[2], so * n[3]);
    W[2 * NG + g] = make_float2(so * n[4], so * n[5]);
}

// ---- averaging ------------------------------------------------------------------------------

__global__ void __launch_bounds__(128) k_fcm_average(int n, const double* __restrict__ r, double L, int N, double h,
                                                     double R_t, float l2s, double wscale,
                                                     const float4* __restrict__ u, double* __restrict__ v) {
    const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    // the blob's box and its offset from the box's first grid point, formed by lane 0 and
    // shared by shuffles: FP64 divisions on every lane would keep the FP64 pipe (1/64 of
    // the FP32 rate) busier than the whole sum over the box
    int lo[3], cn[3];
    float d0[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int l = 0, c = 0;
        float o = 0.f;
        if (lane == 0) {
            double x = r[3LL * i + d];
            x -= L * floor(x / L);
            if (!(x < L) || !(x >= 0.0)) x = 0.0;
            l = (int)ceil((x - R_t) / h);
            c = min(31, (int)floor((x + R_t) / h) - l + 1);
            o = (float)(l * h - x);   // magnitude below R_t + h: FP32 keeps it to ~1e-7 R_t
        }
        lo[d] = __shfl_sync(0xffffffffu, l, 0);
        cn[d] = __shfl_sync(0xffffffffu, c, 0);
        d0[d] = __shfl_sync(0xffffffffu, o, 0);
    }
    // offsets from the blob to the grid points of its box: the first one, then steps of h
    const float hf = (float)h, ih = 1.0f / hf, R2 = (float)(R_t * R_t);
    const float d0x = d0[0], d0y = d0[1], d0z = d0[2];
    const int mask = N - 1;   // N is a power of two
    const int cx = cn[0];
    const float icx = 1.0f / (float)cx;
    // the planes' sums added with compensation (Kahan) in FP32: as accurate as FP64 for a
    // box's at most 31 planes, without an FP32-to-FP64 conversion and FP64 add per plane
    float acc[3] = {0.f, 0.f, 0.f}, cmp[3] = {0.f, 0.f, 0.f};
    float foz = 0.f;   // the plane offset also kept as a float (exact)
    for (int oz = 0; oz < cn[2]; ++oz, foz += 1.f) {
        const float dz = fmaf(foz, hf, d0z), dz2 = dz * dz, rem = R2 - dz2;
        if (rem < 0.f) continue;   // the plane misses the sphere (the same on every lane)
        // the rows that can meet the sphere's disc in this plane (widened by 1% of a row
        // against rounding; the point test decides), taken as one run of points, x fastest,
        // so the lanes stay busy whatever the box width
        const float sq = sqrtf(rem);
        const int y0 = max(0, (int)ceilf((-sq - d0y) * ih - 0.01f));
        const int y1 = min(cn[1] - 1, (int)floorf((sq - d0y) * ih + 0.01f));
        const int npt = (y1 - y0 + 1) * cx;
        const float wz = exp2f(-dz2 * l2s);   // exp(-dz^2 / 2s^2)
        const long long zoff = (long long)((lo[2] + oz) & mask) * N * N;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 4
        for (int p = lane; p < npt; p += 32) {
            // p = (oy - y0) cx + ox; the FP32 quotient is exact (p < 1024, and p / cx lies at
            // least 1 / (2 cx) away from an integer)
            const int qy = (int)(((float)p + 0.5f) * icx);
            const int ox = p - qy * cx, oy = y0 + qy;
            const float dx = fmaf((float)ox, hf, d0x), dy = fmaf((float)oy, hf, d0y);
            const float dxy = fmaf(dx, dx, dy * dy);
            if (dxy + dz2 <= R2) {
                const float wgt = exp2f(-dxy * l2s) * wz;
                const float4 q = __ldg(u + zoff + ((lo[1] + oy) & mask) * N + ((lo[0] + ox) & mask));
                a0 = fmaf(q.x, wgt, a0);
                a1 = fmaf(q.y, wgt, a1);
                a2 = fmaf(q.z, wgt, a2);
            }
        }
        const float a[3] = {a0, a1, a2};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float y = a[c] - cmp[c], t = acc[c] + y;
            cmp[c] = (t - acc[c]) - y;
            acc[c] = t;
        }
    }
    double tot[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        tot[c] = (double)acc[c] - (double)cmp[c];
        for (int o = 16; o > 0; o >>= 1) tot[c] += __shfl_down_sync(0xffffffffu, tot[c], o);
    }
    if (lane == 0) {
        v[3LL * i] = tot[0] * wscale;
        v[3LL * i + 1] = tot[1] * wscale;
        v[3LL * i + 2] = tot[2] * wscale;
    }
}

// ---- host side --------------------------------------------------------------------------------

static gdc_status fcm_fail(gdc_fcm* f, gdc_status s, const std::string& m) {
    if (f) f->err = m;
    return s;
}

static gdc_status fcm_check(gdc_fcm* f, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return GDC_OK;
    return fcm_fail(f, GDC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The transforms along the axes a0 .. a1 - 1 (0 x, 1 y, 2 z) of ncomp grids from slot on.
static void fft3(gdc_fcm* f, int slot, int ncomp, bool inverse, int a0, int a1) {
    float2* d = f->grid + slot * f->NG;
    for (int axis = a0; axis < a1; ++axis) {
        const int th = fft_threads(f->N, axis);
        const dim3 grid((unsigned)(f->NG / (8LL * th)), (unsigned)ncomp);   // N^2 pencils, 8 TH / N per block
        const size_t smem = fft_smem(f->N, th);
#define GDC_FFT(L, TH_)                                                                         \
    do {                                                                                        \
        if (inverse)                                                                            \
            k_fft<1, L, TH_><<<grid, TH_, smem, f->stream>>>(d, f->NG, f->tw, axis);            \
        else                                                                                    \
            k_fft<0, L, TH_><<<grid, TH_, smem, f->stream>>>(d, f->NG, f->tw, axis);            \
    } while (0)
        ++f->n_launch;
        switch (f->logN) {
            case 4: GDC_FFT(4, 256); break;
            case 5: GDC_FFT(5, 256); break;
            case 6: GDC_FFT(6, 256); break;
            case 7: GDC_FFT(7, 256); break;
            case 8:
                if (th == 1024) GDC_FFT(8, 1024);
                else if (th == 512) GDC_FFT(8, 512);
                else GDC_FFT(8, 256);
                break;
            default:
                if (th == 1024) GDC_FFT(9, 1024);
                else if (th == 512) GDC_FFT(9, 512);
                else GDC_FFT(9, 256);
        }
#undef GDC_FFT
    }
}

// The inverse x pass of the velocity in grids slot, slot + 1, packed into packed grid which.
static void fft_x_pack(gdc_fcm* f, int slot, int which) {
    const size_t smem = fft_smem2(f->N, 256);
    const unsigned blocks = (unsigned)(f->NG / (8LL * 256));
    const float2* u = f->grid + slot * f->NG;
    float4* out = f->packed + which * f->NG;
#define GDC_XP(L) k_fft_x_pack<L><<<blocks, 256, smem, f->stream>>>(u, f->NG, f->tw, out)
    ++f->n_launch;
    switch (f->logN) {
        case 4: GDC_XP(4); break;
        case 5: GDC_XP(5); break;
        case 6: GDC_XP(6); break;
        case 7: GDC_XP(7); break;
        case 8: GDC_XP(8); break;
        default: GDC_XP(9);
    }
#undef GDC_XP
}

static void zsolve_launch(gdc_fcm* f) {
    const int th = zsolve_threads(f->N), H = 4 * th / f->N;   // slots (pencil pairs) per block
    const unsigned blocks = (unsigned)ceil_div((long long)f->N * (f->N / 2 + 1), H);
    const size_t smem = fft_smem2(f->N, th);
    const float kunit = (float)(2.0 * 3.141592653589793 / f->p.L);
    const float se = (float)(1.0 / ((double)f->NG * f->p.eta));
    const float2* F = f->grid;
    float2* U = f->grid + 2 * f->NG;
#define GDC_ZS(L, TH_) k_fcm_zsolve<L, TH_><<<blocks, TH_, smem, f->stream>>>(F, U, f->NG, f->tw, kunit, se)
    ++f->n_launch;
    switch (f->logN) {
        case 4: GDC_ZS(4, 256); break;
        case 5: GDC_ZS(5, 256); break;
        case 6: GDC_ZS(6, 256); break;
        case 7: GDC_ZS(7, 256); break;
        case 8: GDC_ZS(8, GDC_ZSOLVE_TH); break;
        default: GDC_ZS(9, GDC_ZSOLVE_TH);
    }
#undef GDC_ZS
}

// which = 0: the deterministic velocity, 1: the fluctuating one
static void fcm_average_launch(gdc_fcm* f, int n, const double* r, int which, double* v) {
    const double s2 = f->p.sigma * f->p.sigma;
    const double norm = std::pow(2.0 * 3.141592653589793 * s2, -1.5);
    ++f->n_launch, k_fcm_average<<<ceil_div(32LL * n, 128), 128, 0, f->stream>>>(
        n, r, f->p.L, f->N, f->h, f->p.R_t, (float)(0.5 / s2 * 1.4426950408889634), norm * f->h * f->h * f->h,
        f->packed + which * f->NG, v);
}

// The grid of a gDC context with the FCM mobility (defaults: sigma = a/sqrt(pi), R_t = 3a).
gdc_fcm_params fcm_params_of(const gdc_params& p, long long n_blobs) {
    gdc_fcm_params f{};
    f.N = p.fcm_N;
    f.L = p.box_L;
    f.sigma = p.fcm_sigma > 0.0 ? p.fcm_sigma : p.a / std::sqrt(3.141592653589793);
    f.R_t = p.fcm_R_t > 0.0 ? p.fcm_R_t : 3.0 * p.a;
    f.eta = p.eta;
    f.max_blobs = (int)std::max(1LL, n_blobs);
    return f;
}

static const char* fcm_args(const gdc_fcm* f, int n, const void* a, const void* b) {
    if (!a || !b) return "NULL pointer";
    if (n < 1 || n > f->p.max_blobs) return "n_blobs must be in [1, max_blobs]";
    return nullptr;
}

}  // namespace gdc

using namespace gdc;

extern "C" {

size_t gdc_fcm_workspace_bytes(const gdc_fcm_params* params) {
    if (fcm_validate(params)) return 0;
    gdc_fcm f;
    fcm_layout(&f, *params);
    return fcm_carve(&f, nullptr);
}

gdc_status gdc_fcm_init(gdc_fcm** out, const gdc_fcm_params* params, void* workspace, size_t ws_bytes, void* stream) {
    if (!out) return GDC_ERR_INVALID_ARG;
    *out = nullptr;
    if (fcm_validate(params) || !workspace) return GDC_ERR_INVALID_ARG;
    gdc_fcm* f = new (std::nothrow) gdc_fcm;
    if (!f) return GDC_ERR_INVALID_ARG;
    fcm_layout(f, *params);
    if (fcm_carve(f, nullptr) > ws_bytes) {
        delete f;
        return GDC_ERR_WORKSPACE;
    }
    fcm_carve(f, workspace);
    f->stream = static_cast<cudaStream_t>(stream);
    std::vector<float2> tw(f->N / 2);
    for (int j = 0; j < f->N / 2; ++j) {
        const double a = 2.0 * 3.141592653589793 * j / f->N;
        tw[j] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    cudaError_t e = cudaMemcpyAsync(f->tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice, f->stream);
    // 1024-thread blocks of 256- and 512-point pencils take 66 and 68 KB of shared memory
    const int fsm = (int)std::max(fft_smem(256, 1024), fft_smem(512, 1024));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft<0, 8, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft<1, 8, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft<0, 9, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft<1, 9, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsm);
    const int zsm = (int)std::max(fft_smem2(256, GDC_ZSOLVE_TH), fft_smem2(512, GDC_ZSOLVE_TH));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fcm_zsolve<8, GDC_ZSOLVE_TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fcm_zsolve<9, GDC_ZSOLVE_TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) {
        delete f;
        return GDC_ERR_CUDA;
    }
    *out = f;
    return GDC_OK;
}

gdc_status gdc_fcm_apply(gdc_fcm* f, int n, const double* r, const double* lambda, double* u) {
    if (!f) return GDC_ERR_INVALID_ARG;
    if (const char* m = fcm_args(f, n, r, lambda)) return fcm_fail(f, GDC_ERR_INVALID_ARG, m);
    if (!u) return fcm_fail(f, GDC_ERR_INVALID_ARG, "NULL pointer");
    const long long nc3 = (long long)f->nc * f->nc * f->nc;
    cudaMemsetAsync(f->cnt, 0, sizeof(int) * nc3, f->stream);
    cudaMemsetAsync(f->fill, 0, sizeof(int) * nc3, f->stream);
    ++f->n_launch, k_fcm_bin<<<ceil_div(n, 256), 256, 0, f->stream>>>(n, r, f->p.L, f->nc, f->pw, f->cell_of, f->cnt);
    scan_exclusive(f->stream, &f->n_launch, (int)nc3, f->cnt, f->start, f->scan);
    ++f->n_launch, k_fcm_scatter<<<ceil_div(n, 256), 256, 0, f->stream>>>(n, f->cell_of, f->start, f->fill, f->list);
    ++f->n_launch, k_cell_sort<<<ceil_div(nc3, 256), 256, 0, f->stream>>>((int)nc3, f->cnt, f->start, f->list);
    ++f->n_launch, k_fcm_stage_blobs<<<ceil_div(n, 256), 256, 0, f->stream>>>(
        n, f->p.L / f->nc, f->nc, f->list, f->cell_of, f->pw, lambda, f->poff, f->plam);
    const double s2 = f->p.sigma * f->p.sigma;
    {
        // 4 grid points per thread, 512 per block (2 and 256 when a cell has at most 256
        // points, so that small cells leave fewer idle slots); the largest cell has side^3 points
        const long long side = (f->N + f->nc - 1) / f->nc;
        const int pt = side * side * side <= 256 ? 2 : 4;
        const unsigned chunks = (unsigned)((side * side * side + 128 * pt - 1) / (128 * pt));
        // the Gaussians as powers of 2: exp(-d^2 / 2s^2) = 2^(-d^2 l2s), l2s = log2(e) / (2 s^2)
        const float R2 = (float)(f->p.R_t * f->p.R_t), i2 = (float)(0.5 / s2 * 1.4426950408889634);
        const float nrm = (float)std::pow(2.0 * 3.141592653589793 * s2, -1.5);
        ++f->n_launch;
#define GDC_SPREAD(PT_, WRAP_)                                                                                      \
    k_fcm_spread<PT_, WRAP_><<<dim3((unsigned)nc3, chunks), 128, 0, f->stream>>>(                                  \
        f->N, f->h, f->p.L, 1.0 / f->p.L, f->p.L / f->nc, f->nc, f->pw, f->cnt, f->start, f->list, lambda, f->poff, \
        f->plam, R2, i2, nrm, f->grid, f->NG)
        const bool wrap = f->nc < 4;
        if (pt == 2) {
            if (wrap)
                GDC_SPREAD(2, true);
            else
                GDC_SPREAD(2, false);
        } else {
            if (wrap)
                GDC_SPREAD(4, true);
            else
                GDC_SPREAD(4, false);
        }
#undef GDC_SPREAD
    }
    // grids 0-1: FFT(f_x + i f_y), FFT(f_z) along x and y; the z passes and the solve in one
    // launch into grids 2-3, the velocity's (u_x + i u_y, u_z); their inverse y pass, then the
    // inverse x pass into packed grid 0
    fft3(f, 0, 2, false, 0, 2);
    zsolve_launch(f);
    fft3(f, 2, 2, true, 1, 2);
    fft_x_pack(f, 2, 0);
    fcm_average_launch(f, n, r, 0, u);
    gdc_status st = fcm_check(f, cudaGetLastError(), "FCM launch");
    if (st == GDC_OK) st = fcm_check(f, cudaStreamSynchronize(f->stream), "FCM product");
    return st;
}

gdc_status gdc_fcm_brownian(gdc_fcm* f, unsigned long long seed, unsigned int owner, unsigned long long step, double kT,
                            double dt, int n, const double* r, double* v) {
    if (!f) return GDC_ERR_INVALID_ARG;
    if (const char* m = fcm_args(f, n, r, v)) return fcm_fail(f, GDC_ERR_INVALID_ARG, m);
    if (!(kT >= 0.0) || !std::isfinite(kT) || !(dt > 0.0) || !std::isfinite(dt))
        return fcm_fail(f, GDC_ERR_INVALID_ARG, "kT must be >= 0 and dt > 0");
    const double dv = f->h * f->h * f->h;
    const double sd = 2.0 * std::sqrt(kT * f->p.eta / (dv * dt)), so = std::sqrt(2.0 * kT * f->p.eta / (dv * dt));
    // grids 4-6: the stress, two real components per complex grid; grids 7-8: (u_x + i u_y, u_z)
    ++f->n_launch, k_fcm_stress<<<ceil_div(f->NG, 256), 256, 0, f->stream>>>(f->NG, seed, owner, step, (float)sd,
                                                                             (float)so, f->grid + 4 * f->NG);
    fft3(f, 4, 3, false, 0, 3);
    ++f->n_launch, k_fcm_solve_stress<<<ceil_div(f->NG, 256), 256, 0, f->stream>>>(
        f->NG, f->N, (float)(2.0 * 3.141592653589793 / f->p.L), (float)(1.0 / ((double)f->NG * f->p.eta)),
        f->grid + 4 * f->NG, f->grid + 7 * f->NG);
    fft3(f, 7, 2, true, 1, 3);
    fft_x_pack(f, 7, 1);
    f->have_field = true;
    fcm_average_launch(f, n, r, 1, v);
    gdc_status st = fcm_check(f, cudaGetLastError(), "FCM launch");
    if (st == GDC_OK) st = fcm_check(f, cudaStreamSynchronize(f->stream), "FCM Brownian velocity");
    return st;
}

gdc_status gdc_fcm_average(gdc_fcm* f, int n, const double* r, double* v) {
    if (!f) return GDC_ERR_INVALID_ARG;
    if (const char* m = fcm_args(f, n, r, v)) return fcm_fail(f, GDC_ERR_INVALID_ARG, m);
    if (!f->have_field) return fcm_fail(f, GDC_ERR_INVALID_ARG, "no fluctuating field yet: call gdc_fcm_brownian first");
    fcm_average_launch(f, n, r, 1, v);
    gdc_status st = fcm_check(f, cudaGetLastError(), "FCM launch");
    if (st == GDC_OK) st = fcm_check(f, cudaStreamSynchronize(f->stream), "FCM average");
    return st;
}

const char* gdc_fcm_last_error(const gdc_fcm* f) { return f ? f->err.c_str() : "NULL context"; }

unsigned long long gdc_fcm_launches(const gdc_fcm* f) { return f ? f->n_launch : 0; }

void gdc_fcm_destroy(gdc_fcm* f) { delete f; }

}  // extern "C"
