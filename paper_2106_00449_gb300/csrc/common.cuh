// Internal definitions shared by the gDC CUDA translation units.
//
// Data layout in device memory (all caller-owned, carved from one workspace):
//   * per suspension s: body range [susp_body_off[s], susp_body_off[s+1]),
//     blob range [susp_blob_off[s], ...), saddle-vector block at susp_gm_off[s]
//     holding [lambda: 3 per blob | V: 6 per body] of that suspension;
//   * blob-indexed vectors (W, v-breve, Lanczos basis) are 3 doubles per blob,
//     global blob order;
//   * body-indexed vectors (V, calV, F) are 6 doubles per body;
//   * the configuration a product is evaluated at ("loaded" configuration):
//     per-body rotation R (9 doubles), per-blob FP64 position r, and the pair
//     kernels' source arrays: float4/double4_32a position relative to the
//     suspension's reference point (w = body index bits) and float4/double4
//     lambda.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gdc.h"

// internal precision of the accurate residual product in FP32-mixed mode: pairs of
// different bodies in double-float arithmetic on the FP32 pipes, same-body blocks in FP64
#define GDC_PREC_DF64 2

#define GDC_MAX_RESTART 100
#define GDC_MAX_LANCZOS 128
#define GDC_MAX_TMPL_BLOBS 340   // 3n <= 1020 rows of a template block
#define GDC_TB_MAX 8             // bodies of one template per block in the factor products
#define GDC_NEAR_CAP 32          // blobs closer than 2a listed per blob (beyond: a search of the suspension)
#define GDC_NEAR_SRC 2048        // sources per block of the near-pair search
#define GDC_SYM_TILE 512         // blobs per tile of the symmetric FP32 pair kernel
#ifndef GDC_DFS_WIDTH
#define GDC_DFS_WIDTH 2          // source tiles per item of the symmetric double-float kernel
#endif
#define GDC_CELL_MIN_BLOBS 16384 // GDC_FORCES_CHOOSE: the cell list from this many blobs on
#define GDC_WAIT_POLLS 400000    // default bound of a pair kernel's wait for a tile copy (polls)

namespace gdc {

struct MvItem {      // one block of the pair kernels: targets [t0, t0+tile) x sources [j0, j1) of suspension s
    int s;
    int t0;          // first target, local to the suspension
    int j0, j1;      // source range, local to the suspension
    int k;           // source-chunk slot of the partial sums
    int pad[3];
};

struct SymItem {     // one block of the symmetric pair kernel: target tile I x source tiles [J0, J1) of suspension s
    int s, I, J0, J1;
    int k;           // target-side partial-sum slot (the item's index within row I)
    int pad[3];
};

struct Chunk {       // a contiguous element range inside one segment, for deterministic reductions
    long long lo, hi;
    int seg;
    int pad;
};

struct Seg {         // a segmented vector space: per-suspension offsets and the chunks covering it
    long long n = 0;           // total length
    const long long* off = 0;  // device, S+1
    std::vector<long long> h_off;
    Chunk* chunks = 0;         // device
    int* seg_chunk_off = 0;    // device, S+1
    std::vector<Chunk> h_chunks;
    std::vector<int> h_seg_chunk_off;
    int n_chunks = 0;
};

// Loop indices of the device-driven Krylov loops (graph mode); lives in the workspace.
struct LoopCtl {
    int lz_j;        // Lanczos iteration index
    int gm_j;        // GMRES inner index within the current cycle
    int gm_total;    // GMRES inner iterations of the current solve
    int gm_checks;   // residual checks of the current solve
    int gm_outer;    // cycles executed (one accurate residual product each)
    int pad[3];
    unsigned long long step;   // step counter the draws use
};

// What one graph-replayed step reports back to the host (one device-to-host read per step).
struct StepReport {
    double lz_err[3];
    double gm_residual;
    double nu_min, nu_max;
    int lz_iters[3];
    int lz_notconv[3];   // stopped at lanczos_max_iter with the change above lanczos_tol
    int lz_exec[3];      // iterations the WHILE node ran
    int gm_total, gm_cycles, gm_converged, gm_bad, gm_notconv, gm_outer;
    int gm_df;           // accurate residual products (the other cycles updated the residual in FP32)
    int status[4];       // copy of the device status words
    int ok;              // 1 when the state was advanced
    int pad;
};

struct Config {      // a rigid configuration the kernels evaluate at
    const double* Y = 0;
    const double* q = 0;
};

}  // namespace gdc

struct gdc_ctx {
    gdc_params p;
    cudaStream_t stream = 0;
    int device = 0, num_sms = 0;
    std::string err;

    // sizes
    int S = 0, NB = 0, NBL = 0, T = 0;
    long long ngm = 0;            // saddle-vector length
    int max_body_blobs = 0;
    unsigned long long step = 0;

    // host copies of the layout
    std::vector<long long> h_body_off, h_blob_off, h_gm_off, h_body_blob_off;
    std::vector<int> h_body_tmpl, h_tmpl_n, h_tmpl_off, h_body_susp;
    // factor products of several bodies of one template per block (body.cu k_body_tri_tb):
    // items (template, first entry in tb_bodies, count), bodies grouped by template
    int4* tb_items = 0;
    int* tb_bodies = 0;
    int tb_n_items = 0;
    bool tb_use = false;   // the grouped products replace one block per body
    size_t tb_smem = 0, tb_precond_smem = 0;
    std::vector<int4> h_tb_items;
    double* lz_qbuf = 0;     // the eigen-step's Q / refined-root scratch per suspension (global)
    bool lz_qbuf_on = false; // more suspensions than SMs: the scratch in global memory, not shared
    std::vector<int> h_tb_bodies;
    std::vector<long long> h_minv_off;
    std::vector<double> h_tmpl_xyz, h_tmpl_L;

    // device layout tables
    long long *susp_body_off = 0, *susp_blob_off = 0, *susp_gm_off = 0, *body_blob_off = 0;
    long long *minv_off = 0;
    int *body_tmpl = 0, *body_susp = 0, *blob_body = 0, *blob_susp = 0, *tmpl_n = 0, *tmpl_off = 0;
    int *blob_gm = 0, *body_gm = 0;
    double *tmpl_xyz = 0, *tmpl_L = 0;
    double *tmpl_Minv = 0, *tmpl_G = 0, *tmpl_N = 0, *tmpl_KtKp = 0, *tmpl_work = 0, *tmpl_M = 0;
    float* tmpl_M32 = 0;          // tmpl_M rounded to FP32 (intra-body block of the FP32 products)
    float* tmpl_Minv32 = 0;       // tmpl_Minv rounded to FP32 (preconditioner of the FP32 inner cycles)
    // factors of the template blocks M_t = L_t L_t^T for the block-preconditioned Lanczos
    // operator, each stored as F with (F-product)_i = sum_k F[k n3 + i] x_k (reads along rows):
    // tmpl_LT = L_t^T (products with L_t), tmpl_X = L_t^-1 (with L_t^-T), tmpl_XT = L_t^-T (with L_t^-1)
    double *tmpl_LT = 0, *tmpl_X = 0, *tmpl_XT = 0;
    float *tmpl_X32 = 0, *tmpl_XT32 = 0;   // L_t^-1 and L_t^-T rounded to FP32 (FP32-mixed Lanczos operator)
    // fluctuating FCM mobility (fcm.cu), GDC_MOB_FCM only
    gdc_fcm* fcm = nullptr;
    double* fcm_u = nullptr;      // M_FCM lambda, 3 per blob
    double* fcm_Mt = nullptr;     // the templates' FCM blocks (preconditioner), like tmpl_M
    void* fcm_ws = nullptr;
    size_t fcm_ws_bytes = 0;
    unsigned long long fcm_field_step = ~0ULL;   // step whose fluctuating field the grid holds
    // cell list of the pair forces (cells.cu)
    long long cell_H = 0;         // buckets: a power of two >= 2 NBL
    int4* cell_xyz = 0;           // per blob: cell coordinates and suspension
    unsigned* cell_key = 0;       // per blob: bucket
    int* cell_cnt = 0;            // per bucket: blobs
    int* cell_start = 0;          // per bucket: first entry of cell_list
    int* cell_fill = 0;           // per bucket: scatter counter
    int* cell_list = 0;           // blob indices grouped by bucket, ascending within a bucket
    int* cell_scan = 0;           // block totals of the bucket-count scan
    double *body_L = 0;

    // state (caller arrays)
    double *Y = 0, *q = 0;

    // loaded configuration
    double *Rb = 0, *r = 0, *Yc = 0, *ref = 0;
    float4 *spos = 0, *slam = 0, *sdup = 0;   // sdup: 3 float4 per blob, pair-kernel tile layout
    double4_32a *spos64 = 0, *slam64 = 0;

    // step buffers
    double *W = 0, *Wt = 0, *vb_n = 0, *vb_t = 0, *vb_m = 0, *calV = 0, *calVt = 0;
    double *Yt = 0, *qt = 0, *Ym = 0, *qm = 0, *FT = 0, *Vm = 0, *nu = 0, *divp = 0, *fblob = 0;
    double *u3 = 0;               // scratch 3 per blob

    // GMRES (saddle layout)
    int m = 0;
    double *gm_V = 0, *gm_x = 0, *gm_b = 0, *gm_r = 0, *gm_w = 0, *gm_z = 0;
    double *gm_H = 0, *gm_cs = 0, *gm_sn = 0, *gm_g = 0, *gm_y = 0, *gm_h = 0, *gm_h2 = 0;
    double *gm_bnorm = 0, *gm_res = 0, *gm_scal = 0;
    int *gm_active = 0, *gm_j = 0;

    // Lanczos (blob layout)
    int kmax = 0;
    double *lz_V = 0, *lz_w = 0, *lz_alpha = 0, *lz_beta = 0, *lz_c = 0;
    double *lz_h = 0, *lz_Wnorm = 0, *lz_err = 0, *lz_scal = 0;
    int *lz_active = 0, *lz_k = 0, *lz_fix = 0, *lz_lastk = 0;
    int* lz_hint = 0;             // per suspension: index the previous unconstrained run stopped at (0 = none)
    double *lz_z = 0, *lz_u = 0;  // preconditioned operator: L^-T x and the product at it (3 per blob)

    // blobs above a wall (gdc_params.wall): per-body blocks set up at every configuration
    std::vector<long long> h_blk_off;          // offsets of the (3 n_p)^2 blocks, NB + 1
    long long* blk_off = 0;
    double *blk_work = 0, *blk_Minv = 0, *blk_G = 0, *blk_N = 0, *blk_LT = 0, *blk_X = 0, *blk_XT = 0;
    std::vector<int2> h_wall_items;            // (suspension, first target) of the wall product
    int2* wall_items = 0;

    // reductions
    gdc::Seg seg_gm, seg_lz, seg_body;
    double* red_part = 0;         // n_chunks x GDC_MAX_LANCZOS partial sums
    int red_cols = 0;

    // pair-kernel work lists
    gdc::MvItem* mv_items = 0;
    int mv_n_items = 0, mv_tpt = 2, mv_threads = 128, mv_kmax = 1;
    int mv_minb = 6;                          // resident blocks per SM the ordered kernel was compiled for (4, 6)
    double mv_waves = 8.0;
    int mv_cap_items = 0, mv_cap_kmax = 1;   // workspace capacity over all autotune candidates
    double autotune_ms = 0.0;                 // best FP32 product time found at init (0 = not tuned)
    int* mv_nk = 0;               // chunks per suspension
    std::vector<gdc::MvItem> h_mv_items;
    std::vector<int> h_mv_nk;
    void* mv_part = 0;            // mv_kmax x NBL x (float4 | double4_32a)
    const int* mv_active = 0;     // when set, suspensions flagged 0 are skipped by the pair kernels

    // symmetric FP32 pair kernel (each unordered pair once) and its work list
    int use_sym = 0, sym_width = 4, sym_n_items = 0, sym_kmax = 1;
    int sym_minb = 2;                         // resident blocks per SM the kernel was compiled for (2, 3, 4)
    int sym_cap_items = 0, sym_cap_kmax = 1;
    long long sym_n_jslots = 0, sym_n_tiles = 0;
    gdc::SymItem* sym_items = 0;
    int* sym_row_nk = 0;                      // target-side slots per tile row
    long long *sym_tile_base = 0, *sym_jbase = 0;   // per suspension: first tile, first source-side slot
    float4 *sym_part_i = 0, *sym_part_j = 0;  // target-side [slot][blob], source-side [slot][GDC_SYM_TILE]
    std::vector<gdc::SymItem> h_sym_items;
    std::vector<int> h_sym_row_nk;
    // symmetric double-float residual kernel (dfsym.cu): its own work list (wider items), FP64 slots
    gdc::SymItem* dfs_items = 0;
    int dfs_n_items = 0, dfs_kmax = 1;
    int dfs_minb = 4;   // 0: the ordered double-float kernel; 3 or 4: symmetric, blocks per SM
    int* dfs_row_nk = 0;
    std::vector<gdc::SymItem> h_dfs_items;
    std::vector<int> h_dfs_row_nk;
    double4_32a *dfs_part_i = 0, *dfs_part_j = 0;
    std::vector<long long> h_sym_tile_base, h_sym_jbase;

    // pairs closer than 2a (self pair excluded) of the loaded configuration, for the FP32
    // products' corrections: per blob a count and up to GDC_NEAR_CAP blob indices
    int4* near_items = 0;         // (suspension, first target, source range) of each search block
    int n_near_items = 0;
    std::vector<int4> h_near_items;
    int *near_cnt = 0, *near_idx = 0;
    double pair_evals_per_matvec = 0.0;

    // host mirrors for convergence checks
    std::vector<int> h_flags;
    std::vector<double> h_vals;

    // optional trace of the last step
    gdc_trace trace{};
    int have_trace = 0;

    // status of device-side loops
    int* dev_status = 0;

    // graph mode: the step replayed as one CUDA graph with WHILE nodes for the Krylov loops
    gdc::LoopCtl* ctl = 0;        // device
    gdc::StepReport* rep = 0;     // device
    double *lz_vcur = 0, *gm_vcur = 0;   // the current Krylov vector, copied out of the basis slot
    cudaGraph_t graph = 0;
    cudaGraphExec_t graph_exec = 0;
    int graph_valid = 0;
    cudaStream_t cap_stream[3] = {0, 0, 0};   // top-level capture, loop body, nested loop body
    cudaStream_t cap_saved[3] = {0, 0, 0};
    cudaGraph_t cap_bodies[2] = {0, 0};        // the two bodies of the IF/ELSE node being captured
    int cap_depth = 0;
    cudaError_t cap_err = cudaSuccess;
    unsigned long long graph_base_launches = 0;               // kernels outside the loops
    std::vector<std::pair<int, unsigned long long>> graph_loops;   // (report slot, kernels per iteration)
    unsigned long long d_step_mirror = ~0ull;                 // value last written to ctl->step

    // instrumentation: kernel launches issued, and CUDA-event timing of the pair kernels
    unsigned long long n_launch = 0;
    int prof_on = 0;
    std::vector<cudaEvent_t> prof_ev;      // start/stop pairs
    std::vector<int> prof_kind;            // 0 = FP32 RPY, 1 = FP64 RPY, 2 = forces, 3 = df64 RPY
    int prof_used = 0;
    double prof_ms[4] = {0, 0, 0, 0};
    unsigned long long prof_count[4] = {0, 0, 0, 0};
};

namespace gdc {

// ---- small device helpers -------------------------------------------------

__host__ __device__ inline void quat_to_R(const double* q, double* R) {
    // Eq. (quaternion_rotation_matrix) of Sec. 2, q scalar first
    const double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    R[0] = 1.0 - 2.0 * q2 * q2 - 2.0 * q3 * q3;
    R[1] = 2.0 * (q1 * q2 - q3 * q0);
    R[2] = 2.0 * (q1 * q3 + q2 * q0);
    R[3] = 2.0 * (q1 * q2 + q3 * q0);
    R[4] = 1.0 - 2.0 * q1 * q1 - 2.0 * q3 * q3;
    R[5] = 2.0 * (q3 * q2 - q1 * q0);
    R[6] = 2.0 * (q1 * q3 - q2 * q0);
    R[7] = 2.0 * (q3 * q2 + q1 * q0);
    R[8] = 1.0 - 2.0 * q2 * q2 - 2.0 * q1 * q1;
}

__device__ inline void quat_exp_mul(const double* u, const double* q, double* out) {
    // out = exp(u) * q: exp of Sec. 2 followed by the Hamilton product of App. A
    const double th = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double s, c;
    if (th < 1e-8) {
        s = 0.5 - th * th / 48.0;      // sin(th/2)/th near 0
        c = cos(0.5 * th);
    } else {
        double sh, ch;
        sincos(0.5 * th, &sh, &ch);
        s = sh / th;
        c = ch;
    }
    const double e0 = c, e1 = s * u[0], e2 = s * u[1], e3 = s * u[2];
    const double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    out[0] = e0 * q0 - (e1 * q1 + e2 * q2 + e3 * q3);
    out[1] = e0 * q1 + q0 * e1 + (e2 * q3 - e3 * q2);
    out[2] = e0 * q2 + q0 * e2 + (e3 * q1 - e1 * q3);
    out[3] = e0 * q3 + q0 * e3 + (e1 * q2 - e2 * q1);
}

__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---- host-side helpers (defined in api.cu) --------------------------------
int first_wait_polls();   // poll bound of the pair kernels' waits for a tile copy (gdc_debug_wait_polls)
gdc_status fail(gdc_ctx* c, gdc_status s, const std::string& msg);
gdc_status cuda_check(gdc_ctx* c, cudaError_t e, const char* what);
int prof_begin(gdc_ctx* c, int kind);     // records a start event when timing is on (-1 otherwise)
void prof_end(gdc_ctx* c, int idx);
void prof_flush(gdc_ctx* c);

// ---- kernels launched across translation units ----------------------------
// geometry.cu
void load_config(gdc_ctx* c, const double* Y, const double* q);
void launch_ref(gdc_ctx* c, const double* Y);
void launch_normals(gdc_ctx* c, unsigned long long step, int stream, double* out,
                    const unsigned long long* step_dev = nullptr);
void launch_perturb(gdc_ctx* c, const double* Y, const double* q, const double* Wt, double delta,
                    double* Yo, double* qo);
void launch_perturb_one(gdc_ctx* c, const double* Y, const double* q, int p_local, int coord,
                        double delta, double* Yo, double* qo);
void launch_advance(gdc_ctx* c, const double* Y, const double* q, const double* V, double h,
                    const double* nu, double* Yo, double* qo, const int* guard = nullptr);
void launch_rfd_div(gdc_ctx* c, const double* Wt, const double* calV, const double* calVt,
                    double delta, double dt, double* nu);
void launch_fd_accum(gdc_ctx* c, const double* calV, const double* calVp, int p_local, int coord,
                     double delta, double* div, int first);
void launch_nu_from_div(gdc_ctx* c, const double* div, double dt, double* nu);
void launch_rhs(gdc_ctx* c, const double* vbrev, const double* FT, double* b);
void launch_scatter_solution(gdc_ctx* c, const double* x, double* V, double* lambda);

// rpy.cu
void launch_pack_lambda(gdc_ctx* c, int prec, const double* x, int gm_layout);
void launch_rpy(gdc_ctx* c, int prec);
void launch_rpy_epilogue(gdc_ctx* c, int prec, const double* x, double* y, int gm_layout,
                         bool same_body = true);   // same_body = false: blocks between different bodies only (FP32)
void launch_forces_pair(gdc_ctx* c, int prec, double* fblob);
void launch_forces_cell(gdc_ctx* c, int prec, double* fblob);
void launch_near_cell(gdc_ctx* c);   // near-pair lists from a cell list (cells.cu)
gdc_fcm_params fcm_params_of(const gdc_params& p, long long n_blobs);
void launch_fcm_saddle_rows(gdc_ctx* c, const double* x, double* y);
void launch_forces(gdc_ctx* c, int prec, double* fblob);   // cell list or all pairs (force_method)
bool forces_use_cells(const gdc_ctx* c);   // pair searches (forces, near pairs) on a cell list
long long cell_buckets(long long NBL);
long long cell_scan_ints(long long NBL);
long long scan_scratch(long long n);   // ints of block totals an exclusive scan of n needs
void scan_exclusive(cudaStream_t st, unsigned long long* n_launch, int n, const int* in, int* out, int* scratch);
__global__ void k_cell_sort(int H, const int* __restrict__ cnt, const int* __restrict__ start, int* __restrict__ list);
void launch_near_build(gdc_ctx* c);
// sym.cu
void build_sym_items(gdc_ctx* c, int width);
void build_sym_list(const gdc_ctx* c, int width, std::vector<SymItem>& items, std::vector<int>& row_nk, int& kmax);
// dfsym.cu
gdc_status dfsym_init_attributes(gdc_ctx* c);
long long lz_q_doubles(int kmax);   // krylov.cu
void launch_rpy_df_sym_pairs(gdc_ctx* c);
void launch_rpy_df_sym_epilogue(gdc_ctx* c, const double* x, double* y, int gm_layout);
gdc_status sym_upload(gdc_ctx* c);
gdc_status sym_init_attributes(gdc_ctx* c);
void launch_rpy32_sym(gdc_ctx* c);
void build_mv_items(gdc_ctx* c, int tpt, double waves);
gdc_status autotune_pair_kernel(gdc_ctx* c);
gdc_status default_pair_kernel(gdc_ctx* c);
void plan_mv_capacity(gdc_ctx* c);
const char* noalloc_last_error();

// body.cu
void launch_body_KT(gdc_ctx* c, const double* x, int x_gm, double* y, int y_gm, double scale);
void launch_lsq(gdc_ctx* c, const double* vbrev, double* calV);
void launch_precond(gdc_ctx* c, const double* r, double* z, bool fp32 = false);
void launch_intra_body(gdc_ctx* c, const double* x, double* y, int gm);
void launch_intra_body32(gdc_ctx* c, const double* x, double* y, int gm);
void launch_template_setup(gdc_ctx* c, const double* Mext = nullptr);   // Mext: given template blocks
// per-body products with the template-block factors L_p = R-hat_p L_t (block-preconditioned
// Lanczos): mode 0 out = L_p^-T x, mode 1 out = L_p^-1 x (+ add), mode 2 out = L_p x
enum { TRI_LINV_T = 0, TRI_LINV = 1, TRI_L = 2 };
void launch_body_tri(gdc_ctx* c, int mode, const double* x, const double* add, double* out, bool fp32 = false);
void launch_wall_blocks(gdc_ctx* c);   // per-body blocks above a wall (at every configuration)

// wall.cu (blobs above a no-slip wall)
void build_wall_items(gdc_ctx* c);
void launch_wall_apply(gdc_ctx* c, int prec, const double* x, double* y, int gm);   // y += W x
void launch_wall_forces(gdc_ctx* c, double* fblob);                                 // fblob += wall + weight

// krylov.cu
gdc_status saddle_op(gdc_ctx* c, int prec, const double* x, double* y);
gdc_status rpy_op(gdc_ctx* c, int prec, const double* lam, double* u);
gdc_status gmres_solve(gdc_ctx* c, const double* b, double* x, gdc_solve_info* info);
gdc_status lanczos_sqrt(gdc_ctx* c, const double* W, double* out, double scale, int fixed_iters,
                        int* iters_out, double* err_out);
void setup_segments(gdc_ctx* c);
void krylov_init_attributes();
// graph mode (capture helpers and the device-driven loops)
cudaGraphConditionalHandle cap_cond(gdc_ctx* c);
void cap_while_begin(gdc_ctx* c, cudaGraphConditionalHandle h);
void cap_while_end(gdc_ctx* c, int report_slot, unsigned long long launches_before);
void lanczos_sqrt_graph(gdc_ctx* c, const double* W, double* out, double scale, int fixed_mode, int run);
void gmres_solve_graph(gdc_ctx* c, const double* b, double* x);
void cap_ifelse_begin(gdc_ctx* c, cudaGraphConditionalHandle h);
void cap_ifelse_next(gdc_ctx* c, int report_slot, unsigned long long launches_before);
void cap_ifelse_end(gdc_ctx* c, int report_slot, unsigned long long launches_before);
// report slots of the loops and branches: Lanczos runs 0..2, GMRES inner iterations, GMRES
// cycles, cycles with an accurate residual product, cycles with an updated residual
enum { REP_LZ0 = 0, REP_GM_TOTAL = 3, REP_GM_OUTER = 4, REP_GM_DF = 5, REP_GM_UPD = 6 };

}  // namespace gdc
