// Fluctuating force-coupling method (FCM) in a periodic cube: M_FCM = J L^-1 S and
// v-breve = J L^-1 D W (Sec. 4.2), discretised as Sec. 4.2 and Sec. 6.1 describe: Gaussian
// envelopes on an N^3 grid cut off beyond R_t, a Fourier spectral Stokes solve, trapezoidal
// averaging, and a fluctuating stress of six independent normals per grid point.
//
// GB300 layout: the grid work is bandwidth-bound, so it runs in FP32 (complex float2 grids,
// nine of N^3 points: 0-2 the deterministic force / velocity, 3-8 the stress, whose last
// three slots end up holding the fluctuating velocity u-breve, kept for re-averaging).
//   * spreading is a gather: each grid point sums the blobs of the 27 periodic binning
//     cells around it (cells at least R_t wide, blobs in ascending index), so it is
//     deterministic and needs no atomics on the grid; distances are formed in FP32 from
//     positions relative to the cells' corners;
//   * the 3-D FFT is three passes of radix-2 transforms of whole pencils in shared memory,
//     16 pencils per block; for the y and z passes the 16 pencils are 16 consecutive x, so
//     every global access is a coalesced run;
//   * the solve (projection, 1/(eta k^2), the spectral divergence of the stress and the 1/N^3
//     of the inverse transform) is one pass over the modes;
//   * averaging takes one warp per blob, lane = x offset inside the blob's box of at most
//     31 grid points per side, with separable Gaussian factors; each lane sums its x column
//     of a z-plane in FP32 and the planes in FP64, and the lanes are added in a fixed order.
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
    float4* prel = nullptr;   // blob positions relative to their binning cell's corner
    int* cell_of = nullptr;
    int* cnt = nullptr;
    int* start = nullptr;
    int* fill = nullptr;
    int* list = nullptr;
    int* scan = nullptr;
    bool have_field = false;
    unsigned long long n_launch = 0;
    std::string err;
};

namespace gdc {

constexpr int FFT_P = 16;     // pencils per FFT block

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
    f->prel = w.take<float4>(f->p.max_blobs);
    f->cell_of = w.take<int>(f->p.max_blobs);
    f->cnt = w.take<int>(nc3);
    f->start = w.take<int>(nc3);
    f->fill = w.take<int>(nc3);
    f->list = w.take<int>(f->p.max_blobs);
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

static size_t fft_smem(int N) { return (size_t)(FFT_P * (N + 1) + N / 2) * sizeof(float2); }

// ---- binning ------------------------------------------------------------------------

// Wraps each blob into the cube, bins it, and keeps its position relative to its binning
// cell's corner in FP32 (small numbers, so FP32 distances stay accurate at any L).
__global__ void k_fcm_bin(int n, const double* __restrict__ r, double L, int nc, float4* __restrict__ prel,
                          int* __restrict__ cell_of, int* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double w = L / nc;
    float x[3];
    int c[3];
    for (int d = 0; d < 3; ++d) {
        double v = r[3LL * i + d];
        v -= L * floor(v / L);
        if (!(v < L) || !(v >= 0.0)) v = 0.0;   // v == L after rounding, or not finite
        c[d] = (int)fmin(fmax(floor(v / w), 0.0), nc - 1.0);
        x[d] = (float)(v - c[d] * w);
    }
    prel[i] = make_float4(x[0], x[1], x[2], 0.f);
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

// f(x_g) = sum of lambda_j Delta_j(x_g) over the blobs of the binning cells around x_g.
// Distances: d = (x_g - corner of its cell) - (p_j - corner of p_j's cell) - o w for the
// cell offset o, all small numbers in FP32; then the minimum image (two comparisons).
__global__ void __launch_bounds__(256) k_fcm_spread(long long NG, int N, double h, double L, int nc,
                                                    const float4* __restrict__ prel, const int* __restrict__ cnt,
                                                    const int* __restrict__ start, const int* __restrict__ list,
                                                    const double* __restrict__ lam, float R2, float inv2s2, float norm,
                                                    float2* __restrict__ f) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= NG) return;
    const double w = L / nc;
    const float wf = (float)w, Lf = (float)L, hL = 0.5f * (float)L;
    const int ig[3] = {(int)(g % N), (int)((g / N) % N), (int)(g / ((long long)N * N))};
    int c[3];
    float xr[3];
    for (int d = 0; d < 3; ++d) {
        const double x = ig[d] * h;
        c[d] = min(nc - 1, (int)(x / w));
        xr[d] = (float)(x - c[d] * w);
    }
    const int no = nc >= 3 ? 3 : nc, o0 = nc >= 3 ? -1 : 0;
    float ax = 0.f, ay = 0.f, az = 0.f;
    for (int oz = 0; oz < no; ++oz)
        for (int oy = 0; oy < no; ++oy)
            for (int ox = 0; ox < no; ++ox) {
                const int o[3] = {o0 + ox, o0 + oy, o0 + oz};
                const int cx = (c[0] + o[0] + nc) % nc, cy = (c[1] + o[1] + nc) % nc, cz = (c[2] + o[2] + nc) % nc;
                const int id = cx + nc * (cy + nc * cz);
                const float bx = xr[0] - o[0] * wf, by = xr[1] - o[1] * wf, bz = xr[2] - o[2] * wf;
                const int e1 = start[id] + cnt[id];
                for (int e = start[id]; e < e1; ++e) {
                    const int j = list[e];
                    const float4 p = prel[j];
                    float dx = bx - p.x, dy = by - p.y, dz = bz - p.z;
                    dx = dx > hL ? dx - Lf : (dx < -hL ? dx + Lf : dx);
                    dy = dy > hL ? dy - Lf : (dy < -hL ? dy + Lf : dy);
                    dz = dz > hL ? dz - Lf : (dz < -hL ? dz + Lf : dz);
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (d2 <= R2) {
                        const float wt = norm * expf(-d2 * inv2s2);
                        ax = fmaf((float)lam[3LL * j], wt, ax);
                        ay = fmaf((float)lam[3LL * j + 1], wt, ay);
                        az = fmaf((float)lam[3LL * j + 2], wt, az);
                    }
                }
            }
    f[g] = make_float2(ax, 0.f);
    f[NG + g] = make_float2(ay, 0.f);
    f[2 * NG + g] = make_float2(az, 0.f);
}

// ---- FFT: radix-2 transforms of 16 pencils per block, one axis per pass -----------------

// INV = 0: X_k = sum_n x_n exp(-2 pi i k n / N); INV = 1: the same with +i, unscaled.
// blockIdx.y picks the component grid (NG points apart).
template <int INV>
__global__ void __launch_bounds__(256) k_fft(float2* __restrict__ data, long long NG, const float2* __restrict__ tw_g,
                                             int N, int logN, int axis) {
    extern __shared__ float2 sm[];
    const int S = N + 1;
    float2* tw = sm + FFT_P * S;
    float2* base = data + blockIdx.y * NG;
    const int groups = N / FFT_P;
    const int b = blockIdx.x;
    long long off, sp, st;   // first element, pencil stride, element stride
    if (axis == 0) {
        off = (long long)N * ((b % groups) * FFT_P + (long long)N * (b / groups));
        sp = N;
        st = 1;
    } else if (axis == 1) {
        off = (b % groups) * FFT_P + (long long)N * N * (b / groups);
        sp = 1;
        st = N;
    } else {
        off = (b % groups) * FFT_P + (long long)N * (b / groups);
        sp = 1;
        st = (long long)N * N;
    }
    for (int j = threadIdx.x; j < N / 2; j += blockDim.x) {
        float2 w = tw_g[j];
        if (INV) w.y = -w.y;
        tw[j] = w;
    }
    const int total = FFT_P * N;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int t = axis == 0 ? e % N : e / FFT_P;
        const int p = axis == 0 ? e / N : e % FFT_P;
        sm[p * S + (int)(__brev((unsigned)t) >> (32 - logN))] = base[off + p * sp + t * st];
    }
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len >> 1, tstep = N / len;
        __syncthreads();
        for (int q = threadIdx.x; q < FFT_P * (N >> 1); q += blockDim.x) {
            const int p = q / (N >> 1), bb = q % (N >> 1);
            const int grp = bb / half, k = bb - grp * half;
            const int i0 = grp * len + k, i1 = i0 + half;
            float2* row = sm + p * S;
            const float2 w = tw[k * tstep];
            const float2 x0 = row[i0], x1 = row[i1];
            const float2 t = make_float2(w.x * x1.x - w.y * x1.y, w.x * x1.y + w.y * x1.x);
            row[i0] = make_float2(x0.x + t.x, x0.y + t.y);
            row[i1] = make_float2(x0.x - t.x, x0.y - t.y);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int t = axis == 0 ? e % N : e / FFT_P;
        const int p = axis == 0 ? e / N : e % FFT_P;
        base[off + p * sp + t * st] = sm[p * S + t];
    }
}

// ---- Fourier-space solve ------------------------------------------------------------------

struct Mode {
    bool keep;
    float kx, ky, kz, k2;
};

__device__ __forceinline__ Mode fcm_mode(long long g, int N, float kunit) {
    const int half = N / 2;
    const int ix = (int)(g % N), iy = (int)((g / N) % N), iz = (int)(g / ((long long)N * N));
    Mode m;
    m.keep = g != 0 && ix != half && iy != half && iz != half;
    m.kx = kunit * (float)(ix < half ? ix : ix - N);
    m.ky = kunit * (float)(iy < half ? iy : iy - N);
    m.kz = kunit * (float)(iz < half ? iz : iz - N);
    m.k2 = m.kx * m.kx + m.ky * m.ky + m.kz * m.kz;
    return m;
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

__global__ void k_fcm_solve(long long NG, int N, float kunit, float scale_eta, float2* __restrict__ u) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= NG) return;
    const Mode m = fcm_mode(g, N, kunit);
    float2 ux = make_float2(0.f, 0.f), uy = ux, uz = ux;
    if (m.keep) fcm_project(m, scale_eta, u[g], u[NG + g], u[2 * NG + g], ux, uy, uz);
    u[g] = ux;
    u[NG + g] = uy;
    u[2 * NG + g] = uz;
}

__device__ __forceinline__ float2 cadd3(float a, float2 x, float b, float2 y, float c, float2 z) {
    return make_float2(a * x.x + b * y.x + c * z.x, a * x.y + b * y.y + c * z.y);
}

// W: the six stress grids (xx, yy, zz, xy, xz, yz); the velocity goes to the last three.
__global__ void k_fcm_solve_stress(long long NG, int N, float kunit, float scale_eta, float2* __restrict__ W) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= NG) return;
    const Mode m = fcm_mode(g, N, kunit);
    float2 ux = make_float2(0.f, 0.f), uy = ux, uz = ux;
    if (m.keep) {
        const float2 xx = W[g], yy = W[NG + g], zz = W[2 * NG + g];
        const float2 xy = W[3 * NG + g], xz = W[4 * NG + g], yz = W[5 * NG + g];
        // (D W)_a = i k_b W_ab
        const float2 dx = cadd3(m.kx, xx, m.ky, xy, m.kz, xz);
        const float2 dy = cadd3(m.kx, xy, m.ky, yy, m.kz, yz);
        const float2 dz = cadd3(m.kx, xz, m.ky, yz, m.kz, zz);
        fcm_project(m, scale_eta, make_float2(-dx.y, dx.x), make_float2(-dy.y, dy.x), make_float2(-dz.y, dz.x), ux, uy,
                    uz);
    }
    W[3 * NG + g] = ux;
    W[4 * NG + g] = uy;
    W[5 * NG + g] = uz;
}

// ---- fluctuating stress ---------------------------------------------------------------------

__global__ void k_fcm_stress(long long NG, unsigned long long seed, unsigned owner, unsigned long long step, double sd,
                             double so, float2* __restrict__ W) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= NG) return;
    const uint2 key = make_uint2((unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
    double n[6];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const uint4 x = philox4x32_10(make_uint4((unsigned)(3 * g + q), owner, (unsigned)(step & 0xffffffffull), 2u), key);
        n[2 * q] = normal_from(x, 0);
        n[2 * q + 1] = normal_from(x, 1);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) W[c * NG + g] = make_float2((float)((c < 3 ? sd : so) * n[c]), 0.f);
}

// ---- averaging ------------------------------------------------------------------------------

__global__ void __launch_bounds__(128) k_fcm_average(int n, const double* __restrict__ r, double L, int N, double h,
                                                     double R_t, float inv2s2, double wscale,
                                                     const float2* __restrict__ u, long long NG, double* __restrict__ v) {
    const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double p[3];
    int lo[3], cn[3];
    for (int d = 0; d < 3; ++d) {
        double x = r[3LL * i + d];
        x -= L * floor(x / L);
        if (!(x < L) || !(x >= 0.0)) x = 0.0;
        p[d] = x;
        lo[d] = (int)ceil((x - R_t) / h);
        cn[d] = min(31, (int)floor((x + R_t) / h) - lo[d] + 1);
    }
    const double R2 = R_t * R_t;
    const bool on = lane < cn[0];
    const int gx = lo[0] + lane;
    const double dx = gx * h - p[0];
    const float wx = on ? expf(-(float)(dx * dx) * inv2s2) : 0.f;
    const int ix = ((gx % N) + N) % N;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int oz = 0; oz < cn[2]; ++oz) {
        const int gz = lo[2] + oz;
        const double dz = gz * h - p[2];
        const float wz = expf(-(float)(dz * dz) * inv2s2);
        const long long zoff = (long long)(((gz % N) + N) % N) * N * N;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int oy = 0; oy < cn[1]; ++oy) {
            const int gy = lo[1] + oy;
            const double dy = gy * h - p[1];
            if (on && dx * dx + dy * dy + dz * dz <= R2) {
                const float w = wx * expf(-(float)(dy * dy) * inv2s2) * wz;
                const long long idx = ix + (long long)(((gy % N) + N) % N) * N + zoff;
                a0 = fmaf(u[idx].x, w, a0);
                a1 = fmaf(u[NG + idx].x, w, a1);
                a2 = fmaf(u[2 * NG + idx].x, w, a2);
            }
        }
        acc[0] += a0;
        acc[1] += a1;
        acc[2] += a2;
    }
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
    if (lane == 0) {
        v[3LL * i] = acc[0] * wscale;
        v[3LL * i + 1] = acc[1] * wscale;
        v[3LL * i + 2] = acc[2] * wscale;
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

static void fft3(gdc_fcm* f, int slot, int ncomp, bool inverse) {
    const dim3 grid((unsigned)(f->N * f->N / FFT_P), (unsigned)ncomp);
    const size_t smem = fft_smem(f->N);
    for (int axis = 0; axis < 3; ++axis) {
        if (inverse)
            ++f->n_launch, k_fft<1><<<grid, 256, smem, f->stream>>>(f->grid + slot * f->NG, f->NG, f->tw, f->N, f->logN, axis);
        else
            ++f->n_launch, k_fft<0><<<grid, 256, smem, f->stream>>>(f->grid + slot * f->NG, f->NG, f->tw, f->N, f->logN, axis);
    }
}

static void fcm_average_launch(gdc_fcm* f, int n, const double* r, int slot, double* v) {
    const double s2 = f->p.sigma * f->p.sigma;
    const double norm = std::pow(2.0 * 3.141592653589793 * s2, -1.5);
    ++f->n_launch, k_fcm_average<<<ceil_div(32LL * n, 128), 128, 0, f->stream>>>(
        n, r, f->p.L, f->N, f->h, f->p.R_t, (float)(0.5 / s2), norm * f->h * f->h * f->h, f->grid + slot * f->NG, f->NG, v);
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
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem(512));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem(512));
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
    ++f->n_launch, k_fcm_bin<<<ceil_div(n, 256), 256, 0, f->stream>>>(n, r, f->p.L, f->nc, f->prel, f->cell_of, f->cnt);
    scan_exclusive(f->stream, &f->n_launch, (int)nc3, f->cnt, f->start, f->scan);
    ++f->n_launch, k_fcm_scatter<<<ceil_div(n, 256), 256, 0, f->stream>>>(n, f->cell_of, f->start, f->fill, f->list);
    ++f->n_launch, k_cell_sort<<<ceil_div(nc3, 256), 256, 0, f->stream>>>((int)nc3, f->cnt, f->start, f->list);
    const double s2 = f->p.sigma * f->p.sigma;
    ++f->n_launch, k_fcm_spread<<<ceil_div(f->NG, 256), 256, 0, f->stream>>>(
        f->NG, f->N, f->h, f->p.L, f->nc, f->prel, f->cnt, f->start, f->list, lambda, (float)(f->p.R_t * f->p.R_t),
        (float)(0.5 / s2),
        (float)std::pow(2.0 * 3.141592653589793 * s2, -1.5), f->grid);
    fft3(f, 0, 3, false);
    ++f->n_launch, k_fcm_solve<<<ceil_div(f->NG, 256), 256, 0, f->stream>>>(
        f->NG, f->N, (float)(2.0 * 3.141592653589793 / f->p.L), (float)(1.0 / ((double)f->NG * f->p.eta)), f->grid);
    fft3(f, 0, 3, true);
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
    ++f->n_launch, k_fcm_stress<<<ceil_div(f->NG, 256), 256, 0, f->stream>>>(f->NG, seed, owner, step, sd, so,
                                                                             f->grid + 3 * f->NG);
    fft3(f, 3, 6, false);
    ++f->n_launch, k_fcm_solve_stress<<<ceil_div(f->NG, 256), 256, 0, f->stream>>>(
        f->NG, f->N, (float)(2.0 * 3.141592653589793 / f->p.L), (float)(1.0 / ((double)f->NG * f->p.eta)),
        f->grid + 3 * f->NG);
    fft3(f, 6, 3, true);
    f->have_field = true;
    fcm_average_launch(f, n, r, 6, v);
    gdc_status st = fcm_check(f, cudaGetLastError(), "FCM launch");
    if (st == GDC_OK) st = fcm_check(f, cudaStreamSynchronize(f->stream), "FCM Brownian velocity");
    return st;
}

gdc_status gdc_fcm_average(gdc_fcm* f, int n, const double* r, double* v) {
    if (!f) return GDC_ERR_INVALID_ARG;
    if (const char* m = fcm_args(f, n, r, v)) return fcm_fail(f, GDC_ERR_INVALID_ARG, m);
    if (!f->have_field) return fcm_fail(f, GDC_ERR_INVALID_ARG, "no fluctuating field yet: call gdc_fcm_brownian first");
    fcm_average_launch(f, n, r, 6, v);
    gdc_status st = fcm_check(f, cudaGetLastError(), "FCM launch");
    if (st == GDC_OK) st = fcm_check(f, cudaStreamSynchronize(f->stream), "FCM average");
    return st;
}

const char* gdc_fcm_last_error(const gdc_fcm* f) { return f ? f->err.c_str() : "NULL context"; }

unsigned long long gdc_fcm_launches(const gdc_fcm* f) { return f ? f->n_launch : 0; }

void gdc_fcm_destroy(gdc_fcm* f) { delete f; }

}  // extern "C"
