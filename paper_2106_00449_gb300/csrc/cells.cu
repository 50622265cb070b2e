// Cell list for the short-range pair forces between blobs of different bodies.
//
// The pair force vanishes (below 1e-15 of its scale) beyond the cutoff r_c, so blob i
// only needs the blobs of the 27 cells around its own when cells are at least r_c wide:
// O(N_b) work at bounded density instead of the N_b^2 of the all-pairs tiles.  The domain
// is unbounded and bodies drift, so cells are not stored as a grid: the integer cell
// coordinates (and the suspension) are hashed into H buckets, H a power of two of at least
// 2 N_b, and a bucket lists its blobs in ascending index.  A bucket may hold blobs of
// several cells (hash collisions); a blob is taken only when its own cell is the
// neighbour cell being visited, so every pair is seen exactly once per direction.
//
// Build (every configuration): cell and bucket per blob with a count per bucket; an
// exclusive scan of the counts; a scatter into the buckets; an insertion sort of each
// bucket by blob index.  The scatter order is arbitrary, the sorted lists are not, and
// each blob sums its terms cell by cell in a fixed order: the forces are deterministic.
#include <algorithm>

#include "common.cuh"
#include "forces.cuh"

namespace gdc {

constexpr int SCAN_B = 1024;

__device__ __forceinline__ unsigned cell_hash(int ix, int iy, int iz, int s, unsigned mask) {
    return ((unsigned)ix * 73856093u ^ (unsigned)iy * 19349663u ^ (unsigned)iz * 83492791u ^ (unsigned)s * 2654435761u) &
           mask;
}

// floor(x / h) as an int, clamped so that a wild coordinate cannot overflow the cast
__device__ __forceinline__ int cell_coord(double x, double h_inv) {
    const double v = fmin(fmax(floor(x * h_inv), -1073741824.0), 1073741823.0);
    return (int)v;
}

// Cells of the blobs.  box > 0 (a periodic cube, the FCM mobility): positions r wrapped into
// the cube, nc cells of side box / nc per axis; otherwise cells of side 1 / h_inv from the
// positions relative to the suspension's reference point.
__global__ void k_cell_assign(int NBL, const double4_32a* __restrict__ spos64, const double* __restrict__ r,
                              const int* __restrict__ blob_susp, double h_inv, double box, int nc, unsigned mask,
                              int4* __restrict__ cell_xyz, unsigned* __restrict__ cell_key, int* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const int s = blob_susp[i];
    int4 cc;
    if (box > 0.0) {
        int c[3];
        for (int d = 0; d < 3; ++d) {
            double v = r[3LL * i + d];
            v -= box * floor(v / box);
            c[d] = (int)fmin(fmax(floor(v * nc / box), 0.0), nc - 1.0);
        }
        cc = make_int4(c[0], c[1], c[2], s);
    } else {
        const double4_32a p = spos64[i];
        cc = make_int4(cell_coord(p.x, h_inv), cell_coord(p.y, h_inv), cell_coord(p.z, h_inv), s);
    }
    const unsigned key = cell_hash(cc.x, cc.y, cc.z, s, mask);
    cell_xyz[i] = cc;
    cell_key[i] = key;
    atomicAdd(cnt + key, 1);
}

// Exclusive scan of in[0, n) within blocks of SCAN_B elements; block totals to tot.
__global__ void __launch_bounds__(SCAN_B) k_scan_block(int n, const int* __restrict__ in, int* __restrict__ out,
                                                       int* __restrict__ tot) {
    __shared__ int wsum[SCAN_B / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long i = (long long)blockIdx.x * SCAN_B + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const int excl = x - v + (warp > 0 ? wsum[warp - 1] : 0);
    if (i < n) out[i] = excl;
    if (threadIdx.x == SCAN_B - 1) tot[blockIdx.x] = excl + v;
}

__global__ void k_scan_add(int n, int* __restrict__ out, const int* __restrict__ base) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += base[i / SCAN_B];
}

// Scratch ints the scan of n elements needs for its block totals (all levels).
long long scan_scratch(long long n) {
    long long s = 0;
    while (n > 1) {
        n = (n + SCAN_B - 1) / SCAN_B;
        s += 2 * n;
    }
    return s + 2;
}

// out = exclusive scan of in[0, n), with the block totals of every level in scratch
// (scan_scratch(n) ints); kernels counted in *n_launch
void scan_exclusive(cudaStream_t st, unsigned long long* n_launch, int n, const int* in, int* out, int* scratch) {
    const int nb = ceil_div(n, SCAN_B);
    int* tot = scratch;
    ++*n_launch, k_scan_block<<<nb, SCAN_B, 0, st>>>(n, in, out, tot);
    if (nb == 1) return;
    int* tot_ex = scratch + nb;
    scan_exclusive(st, n_launch, nb, tot, tot_ex, scratch + 2 * nb);
    ++*n_launch, k_scan_add<<<ceil_div(n, 256), 256, 0, st>>>(n, out, tot_ex);
}

static void scan_exclusive(gdc_ctx* c, int n, const int* in, int* out, int* scratch) {
    scan_exclusive(c->stream, &c->n_launch, n, in, out, scratch);
}

__global__ void k_cell_scatter(int NBL, const unsigned* __restrict__ cell_key, const int* __restrict__ start,
                               int* __restrict__ fill, int* __restrict__ list) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const unsigned key = cell_key[i];
    list[start[key] + atomicAdd(fill + key, 1)] = i;
}

__global__ void k_cell_sort(int H, const int* __restrict__ cnt, const int* __restrict__ start, int* __restrict__ list) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= H) return;
    const int n = cnt[b];
    if (n < 2) return;
    int* l = list + start[b];
    for (int i = 1; i < n; ++i) {
        const int v = l[i];
        int j = i - 1;
        while (j >= 0 && l[j] > v) {
            l[j + 1] = l[j];
            --j;
        }
        l[j + 1] = v;
    }
}

__device__ __forceinline__ long long body_of(float4 p) { return __float_as_int(p.w); }
__device__ __forceinline__ long long body_of(double4_32a p) { return (long long)p.w; }

// f_i = sum over blobs j of other bodies within the cutoff of F(r_ij) (r_i - r_j)/r_ij, in
// precision T from the pair kernels' positions (relative to the suspension's reference
// point); neighbour cells in z, y, x order, each bucket in ascending blob index.
// box > 0: a periodic cube of nc >= 3 cells per axis; neighbour cells wrap and distances
// are minimum images.
template <typename T, typename P4>
__global__ void __launch_bounds__(128) k_forces_cell(int NBL, const P4* __restrict__ pos, const int4* __restrict__ cell_xyz,
                                                     const int* __restrict__ cnt, const int* __restrict__ start,
                                                     const int* __restrict__ list, unsigned mask, ForceK<T> k,
                                                     T box, int nc, double* __restrict__ fblob) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const P4 pi = pos[i];
    const long long bi = body_of(pi);
    const int4 ci = cell_xyz[i];
    T fx = T(0), fy = T(0), fz = T(0);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int cx = ci.x + dx, cy = ci.y + dy, cz = ci.z + dz;
                if (box > T(0)) {
                    cx = (cx + nc) % nc;
                    cy = (cy + nc) % nc;
                    cz = (cz + nc) % nc;
                }
                const unsigned key = cell_hash(cx, cy, cz, ci.w, mask);
                const int e0 = start[key], e1 = e0 + cnt[key];
                for (int e = e0; e < e1; ++e) {
                    const int j = list[e];
                    const int4 cj = cell_xyz[j];
                    if (cj.x != cx || cj.y != cy || cj.z != cz || cj.w != ci.w) continue;
                    const P4 pj = pos[j];
                    T ddx = pi.x - pj.x, ddy = pi.y - pj.y, ddz = pi.z - pj.z;
                    if (box > T(0)) {
                        ddx -= box * rint(ddx / box);
                        ddy -= box * rint(ddy / box);
                        ddz -= box * rint(ddz / box);
                    }
                    const T r2 = fma(ddx, ddx, fma(ddy, ddy, ddz * ddz));
                    if (body_of(pj) != bi && r2 < k.rc2 && r2 > T(0)) {
                        const T r = sqrt(r2);
                        const T s = pair_force(r, k) / r;
                        fx = fma(s, ddx, fx);
                        fy = fma(s, ddy, fy);
                        fz = fma(s, ddz, fz);
                    }
                }
            }
    fblob[3LL * i] = (double)fx;
    fblob[3LL * i + 1] = (double)fy;
    fblob[3LL * i + 2] = (double)fz;
}

long long cell_buckets(long long NBL) {
    long long H = 1024;
    while (H < 2 * NBL) H *= 2;
    return H;
}

long long cell_scan_ints(long long NBL) { return scan_scratch(cell_buckets(NBL)); }

bool forces_use_cells(const gdc_ctx* c) {
    return c->p.mobility == GDC_MOB_FCM || c->p.force_method == GDC_FORCES_CELL_LIST ||
           (c->p.force_method == GDC_FORCES_CHOOSE && c->NBL >= GDC_CELL_MIN_BLOBS);
}

// Periodic cells of the FCM cube for the pair forces: as many per axis as fit at least the
// cutoff (with margin); validation requires 3 or more.
static int periodic_cells(const gdc_ctx* c) {
    return (int)std::floor(c->p.box_L / (force_cutoff(c->p) * (1.0 + 1e-4)));
}

// For every blob i, the blobs j of other bodies of its suspension whose FP32 r_ij^2, formed
// with the FP32 pair kernels' operations (source minus target, fma(dx, dx, fma(dy, dy,
// dz dz))), is below 4a^2, from a cell list of cells at least 2a wide: the list k_near_build
// makes from every pair, entry for entry (k_near_sort then orders both the same way).
__global__ void __launch_bounds__(128) k_near_cell(int NBL, const float4* __restrict__ spos,
                                                   const int4* __restrict__ cell_xyz, const int* __restrict__ cnt,
                                                   const int* __restrict__ start, const int* __restrict__ list,
                                                   unsigned mask, float four_a2, int* __restrict__ near_cnt,
                                                   int* __restrict__ near_idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NBL) return;
    const float4 pi = spos[i];
    const int4 ci = cell_xyz[i];
    int m = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int cx = ci.x + dx, cy = ci.y + dy, cz = ci.z + dz;
                const unsigned key = cell_hash(cx, cy, cz, ci.w, mask);
                const int e0 = start[key], e1 = e0 + cnt[key];
                for (int e = e0; e < e1; ++e) {
                    const int j = list[e];
                    const int4 cj = cell_xyz[j];
                    if (cj.x != cx || cj.y != cy || cj.z != cz || cj.w != ci.w) continue;
                    const float4 pj = spos[j];
                    const float ddx = __fsub_rn(pj.x, pi.x), ddy = __fsub_rn(pj.y, pi.y), ddz = __fsub_rn(pj.z, pi.z);
                    const float r2 = __fmaf_rn(ddx, ddx, __fmaf_rn(ddy, ddy, __fmul_rn(ddz, ddz)));
                    if (r2 < four_a2 && __float_as_int(pj.w) != __float_as_int(pi.w)) {
                        if (m < GDC_NEAR_CAP) near_idx[(long long)i * GDC_NEAR_CAP + m] = j;
                        ++m;
                    }
                }
            }
    near_cnt[i] = m;
}

// Buckets of the cells of edge h, or of nc periodic cells per axis of a cube of side box > 0
// (bucket counts, starts and blob lists, sorted within a bucket).
static void build_cells(gdc_ctx* c, double h, double box = 0.0, int nc = 0) {
    const int H = (int)c->cell_H;
    const unsigned mask = (unsigned)(H - 1);
    cudaMemsetAsync(c->cell_cnt, 0, sizeof(int) * H, c->stream);
    cudaMemsetAsync(c->cell_fill, 0, sizeof(int) * H, c->stream);
    ++c->n_launch, k_cell_assign<<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(
        c->NBL, c->spos64, c->r, c->blob_susp, 1.0 / h, box, nc, mask, c->cell_xyz, c->cell_key, c->cell_cnt);
    scan_exclusive(c, H, c->cell_cnt, c->cell_start, c->cell_scan);
    ++c->n_launch, k_cell_scatter<<<ceil_div(c->NBL, 256), 256, 0, c->stream>>>(c->NBL, c->cell_key, c->cell_start,
                                                                                c->cell_fill, c->cell_list);
    ++c->n_launch, k_cell_sort<<<ceil_div(H, 256), 256, 0, c->stream>>>(H, c->cell_cnt, c->cell_start, c->cell_list);
}

void launch_near_cell(gdc_ctx* c) {
    // cells 2a wide (and a margin): an FP32 r^2 below 4a^2 stays within adjacent cells
    build_cells(c, 2.0 * c->p.a * (1.0 + 1e-4));
    ++c->n_launch, k_near_cell<<<ceil_div(c->NBL, 128), 128, 0, c->stream>>>(
        c->NBL, c->spos, c->cell_xyz, c->cell_cnt, c->cell_start, c->cell_list, (unsigned)(c->cell_H - 1),
        (float)(4.0 * c->p.a * c->p.a), c->near_cnt, c->near_idx);
}

void launch_forces_cell(gdc_ctx* c, int prec, double* fblob) {
    const unsigned mask = (unsigned)(c->cell_H - 1);
    const int pe = prof_begin(c, 2);
    const bool periodic = c->p.mobility == GDC_MOB_FCM;
    const double box = periodic ? c->p.box_L : 0.0;
    const int nc = periodic ? periodic_cells(c) : 0;
    build_cells(c, force_cutoff(c->p) * (1.0 + 1e-4), box, nc);   // FP32 r^2 < r_c^2 stays within adjacent cells
    if (prec == GDC_FP32_MIXED)
        ++c->n_launch, k_forces_cell<float, float4><<<ceil_div(c->NBL, 128), 128, 0, c->stream>>>(
            c->NBL, c->spos, c->cell_xyz, c->cell_cnt, c->cell_start, c->cell_list, mask, force_constants<float>(c->p),
            (float)box, nc, fblob);
    else
        ++c->n_launch, k_forces_cell<double, double4_32a><<<ceil_div(c->NBL, 128), 128, 0, c->stream>>>(
            c->NBL, c->spos64, c->cell_xyz, c->cell_cnt, c->cell_start, c->cell_list, mask, force_constants<double>(c->p),
            box, nc, fblob);
    prof_end(c, pe);
}

void launch_forces(gdc_ctx* c, int prec, double* fblob) {
    if (forces_use_cells(c))
        launch_forces_cell(c, prec, fblob);
    else
        launch_forces_pair(c, prec, fblob);
}

}  // namespace gdc
