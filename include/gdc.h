/*
 * gdc.h -- C ABI of the GB300 library for the generalised drift-correcting
 * (gDC) time step of Brownian suspensions of rigid multiblob bodies
 * (Westwood, Delmotte & Keaveny, arXiv 2106.00449).
 *
 * Model (Sec. 2): N rigid bodies, body p at centre Y_p with unit quaternion
 * q_p = (q0, q1, q2, q3) (scalar first, App. A), made of blobs of radius a
 * placed at r_i = Y_p + R(q_p) b_i (Eq. quaternion_rotation_matrix).  Blobs interact through the
 * unbounded Rotne-Prager-Yamakawa tensor including its overlapping-blob form
 * (Sec. 4.1).  lambda (3 per blob) is the force a blob exerts on the fluid
 * (Eq. ddof_mob); V_p = [Ydot_p, Omega_p] (Sec. 2.2); F_p = [force; torque].
 *
 * Memory.  Every array argument named "dev" is device memory owned by the
 * caller; every "host" array is host memory owned by the caller.  The
 * library allocates no device memory: the caller passes one workspace of
 * gdc_workspace_bytes() bytes to gdc_init and keeps it alive until
 * gdc_destroy.  All work is issued on the stream given to gdc_init, in
 * order; calls that return info structs synchronise that stream first.
 *
 * Batching.  One context holds S independent suspensions.  Bodies are
 * numbered suspension by suspension (susp_body_off), blobs body by body in
 * template order.  Suspensions never interact; each has its own nu, its
 * own Krylov spaces and its own random stream.
 *
 * Errors.  Every call returns a gdc_status; a non-OK status leaves a one-line
 * description in gdc_last_error(ctx).  Invalid sizes, non-unit quaternions,
 * a too-small workspace and out-of-range parameters are rejected on the
 * host before any launch.  Nothing aborts, traps or hangs: Krylov loops stop
 * at their iteration limits and report GDC_ERR_NOT_CONVERGED, non-finite
 * results report GDC_ERR_NONFINITE.
 */
#ifndef GDC_H
#define GDC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GDC_OK = 0,
    GDC_ERR_INVALID_ARG = 1,
    GDC_ERR_CUDA = 2,
    GDC_ERR_NOT_CONVERGED = 3,
    GDC_ERR_NONFINITE = 4,
    GDC_ERR_TIMEOUT = 5,
    GDC_ERR_WORKSPACE = 6
} gdc_status;

/* Precision of the O(N_b^2) pair evaluations.  GDC_FP64: everything in FP64.
 * GDC_FP32_MIXED: pair kernels in FP32 (FP64 across tiles); Krylov
 * recurrences, the preconditioner and the state in FP64; the mobility solve
 * restarts from an FP64 residual until that residual meets gmres_tol. */
typedef enum { GDC_FP64 = 0, GDC_FP32_MIXED = 1 } gdc_precision;

/* Precision of the accurate product that GDC_FP32_MIXED checks its residuals with,
 * accepted by gdc_rpy_apply / gdc_saddle_apply: pairs of different bodies in
 * double-float arithmetic (two floats, about 48 significant bits) on the FP32 pipes,
 * same-body blocks in FP64. */
#define GDC_DF64_RESIDUAL 2

/* Divergence estimate of Sec. 3 step 3: random finite differences (Eq. rfd_div)
 * or finite differences over every body coordinate (Eq. FD). */
typedef enum { GDC_DIV_RFD = 0, GDC_DIV_FD = 1 } gdc_divmode;

/* Time integrator: the gDC of Sec. 3, or Euler-Maruyama of App. D (no drift). */
typedef enum { GDC_SCHEME_GDC = 0, GDC_SCHEME_EM = 1 } gdc_scheme;

/* Mobility of the blobs: the unbounded RPY tensor (Sec. 4.1), or the fluctuating FCM of
 * Sec. 4.2 in a periodic cube (one suspension; pair forces at minimum-image distances on a
 * periodic cell list, which needs box_L of at least 3 force cutoffs).  With FCM the Brownian
 * slip of a step is J u-breve for one fluctuating field u-breve = L^-1 D W drawn at the
 * step's start (stress of (seed, 0, step), see gdc_fcm_*) and averaged again at every later
 * configuration of the step -- the perturbed states of step 3 and the mid-step (Sec. 5);
 * the RPY-only settings (Lanczos tolerances, pair kernels) are not used, all products use
 * the FP32-grid FCM operator whatever the precision (GMRES then runs without refinement
 * cycles and counts its products as matvecs_fp64; relative rounding a few 1e-7, so
 * gmres_tol should be 1e-5 or looser; Sec. 6.2 uses 1e-4), the block preconditioner uses
 * each template's FCM block (computed at init from 3 n_t FCM products), and steps run
 * host-driven. */
typedef enum { GDC_MOB_RPY = 0, GDC_MOB_FCM = 1 } gdc_mobility;

/* Pair potential between blobs of different bodies (the forces F^m of Sec. 3 step 4):
 * the soft sphere U of Eq. soft_sphere_potential alone, or with the Gaussian wells
 * phi_c(r) = A_w exp(-((r - c)/lambda)^2) of Sec. 6.4: U_1 = U - phi_3a (repel-attract)
 * or U_2 = U - phi_3a + phi_7a/2 (repel-attract-repel).  Each continues linearly below
 * r = 2a, so overlapping blobs feel the force at 2a. */
typedef enum { GDC_POT_SOFT = 0, GDC_POT_REPEL_ATTRACT = 1, GDC_POT_REPEL_ATTRACT_REPEL = 2 } gdc_potential;

/* How the short-range pair searches run -- the pair forces, and the list of pairs of
 * different bodies closer than 2a that the FP32 RPY products correct: every pair of a
 * suspension in tiles, or a cell list whose cells are at least the search radius wide
 * (O(N_b) work at bounded density).  Both give the same pairs; the near-pair lists are
 * identical entry for entry, so FP32 products do not depend on the method. */
typedef enum { GDC_FORCES_CHOOSE = 0, GDC_FORCES_ALL_PAIRS = 1, GDC_FORCES_CELL_LIST = 2 } gdc_force_method;

typedef struct {
    double eta;            /* fluid viscosity (Sec. 4.2)                               */
    double kT;             /* thermal energy k_B T (Eq. system_sde)                             */
    double a;              /* blob radius (Sec. 4.1)                                   */
    double dt;             /* time step Delta t (Sec. 3)                               */
    double gmres_tol;      /* relative residual of the mobility solve (Sec. 2.2, 5)   */
    int    gmres_max_iter; /* total inner GMRES iterations allowed per solve           */
    int    gmres_restart;  /* Krylov basis size per cycle, 2..100                      */
    double lanczos_tol;    /* relative change of M^(1/2) W between iterations (Sec. 4.1) */
    int    lanczos_max_iter; /* 2..128                                                */
    double rfd_delta;      /* delta of Eqs. FD and rfd_div (Sec. 6.2 uses 1e-6)                 */
    int    precision;      /* gdc_precision                                            */
    int    divmode;        /* gdc_divmode                                              */
    int    scheme;         /* gdc_scheme                                               */
    double rep_A;          /* soft repulsion amplitude A (force units), 0 = off        */
    double rep_b;          /* soft repulsion range b (Eq. soft_sphere_potential)                          */
    double shear_rate;     /* background flow u = (shear_rate * y, 0, 0); 0 = off      */
    unsigned long long seed; /* Philox4x32-10 key of the W and W-tilde draws            */
    int    autotune;       /* 1: gdc_init times the FP32 pair kernels' candidates at the
                              initial configuration and keeps the fastest: kernel, work-
                              item shape and the resident blocks per SM it is compiled for;
                              then the double-float residual kernels (ordered, symmetric
                              at 3 or 4 blocks per SM) the same way                      */
    int    graph;          /* 1: gdc_step captures one step as a CUDA graph at its first
                              call and replays it; the Lanczos and GMRES loops are
                              conditional WHILE nodes whose conditions the loop kernels
                              set, so a step makes one device-to-host read instead of one
                              per Krylov iteration.  Results are identical to graph = 0
                              (host-driven loops).  Used for the RFD divergence and for
                              Euler-Maruyama, not while gdc_profile is on.              */
    int    pair_kernel;    /* FP32 RPY pair kernel, fixed at init: 1 ordered (every ordered
                              pair, target-side sums), 2 symmetric (every unordered pair
                              once, both sides), 0 the faster of the two as timed by the
                              autotuner (symmetric when autotune = 0).  The double-float
                              residual kernel is ordered for 1, symmetric for 2, and for
                              0 the autotuner's pick (symmetric when autotune = 0)        */
    int    potential;      /* gdc_potential                                            */
    double well_A;         /* well amplitude A_w, energy units (Sec. 6.4: 5 kT); 0 = no wells */
    double well_lambda;    /* well width lambda, a length (Sec. 6.4: 0.5 a)            */
    int    force_method;   /* gdc_force_method; GDC_FORCES_CHOOSE takes the cell list from
                              16,384 blobs on and every pair below.  Both sum the pairs
                              closer than the cutoff (36 b past 2a for the soft sphere,
                              6 lambda past the outer well centre), each blob's terms in
                              a fixed order: results are deterministic.                 */
    int    mobility;       /* gdc_mobility                                             */
    double box_L;          /* GDC_MOB_FCM: side of the periodic cube                   */
    int    fcm_N;          /* GDC_MOB_FCM: grid points per side (power of two, 16..512)  */
    double fcm_sigma;      /* GDC_MOB_FCM: envelope width; 0 = a / sqrt(pi)             */
    double fcm_R_t;        /* GDC_MOB_FCM: envelope truncation radius; 0 = 3a          */
    int    lanczos_precond; /* M^(1/2) W by Lanczos (Sec. 4.1): 1 builds the Krylov space of the
                              block-preconditioned operator A = L^-1 M L^-T of Chow & Saad, with
                              L = diag_p(R(q_p)-hat L_t) and L_t the Cholesky factor of the
                              template's RPY block (L L^T = the body blocks of M), and
                              returns L A^(1/2) W; 0 uses M itself and returns its symmetric
                              root M^(1/2) W.  Both roots S satisfy S S^T = M, so v-breve has
                              the covariance (2 kT / dt) M either way; 1 needs fewer products */
    int    wall;           /* 1: the blobs move above a no-slip wall at z = 0 (the setting of the
                              paper's RPY runs, Sec. 4.1 and 6.2): M is the RPY tensor plus its
                              wall correction (the Rotne-Prager regularisation of the image system
                              of a point force above a wall), every blob centre must stay above
                              z = a (a blob reaching it stops the call with GDC_ERR_NONFINITE and
                              leaves the state unchanged), and the per-body blocks of both
                              preconditioners are set up for each body at every configuration
                              (FP64 Cholesky per body); RPY mobility only, no background shear */
    double wall_V0;        /* with wall: every blob at height h feels -dV/dh of
                              V(h) = wall_V0 a exp(-(h - a)/wall_b) / (h - a) (Sec. 6.2: 23 kT) */
    double wall_b;         /* its range, a length (Sec. 6.2: 0.5 a)                    */
    double body_weight;    /* with wall: a force body_weight along -z on every body, shared
                              equally by its blobs (Sec. 6.2: mg = 0.18 kT/a)            */
    int    df_kernel;      /* double-float residual kernel, fixed at init: 0 as pair_kernel
                              says, 1 ordered, 3 or 4 symmetric compiled for that many
                              resident blocks per SM; all give the same product up to
                              summation order                                           */
} gdc_params;

typedef struct {
    int    iterations;     /* inner GMRES iterations (largest over suspensions)        */
    int    cycles;         /* restart / refinement cycles                              */
    int    matvecs_fp32;   /* RPY products evaluated in FP32                           */
    int    matvecs_fp64;   /* RPY products evaluated in FP64                           */
    double residual;       /* largest relative FP64 residual ||b - A x|| / ||b||        */
    int    converged;      /* 1 when every suspension met gmres_tol                    */
} gdc_solve_info;

typedef struct {
    unsigned long long step;      /* step counter the draws of this step used          */
    int    lanczos_iters[3];      /* at x^n, at x^n + delta W~ (or all FD states), at x^m */
    double lanczos_err;           /* largest final Lanczos change estimate             */
    gdc_solve_info solve;         /* the mid-step mobility solve (Sec. 3 step 5)       */
    double nu_min, nu_max;        /* range of nu over suspensions (Sec. 3 step 3)      */
    double pair_evals;            /* ordered blob pairs evaluated by RPY products      */
} gdc_step_info;

/* Device pointers that gdc_step fills with the intermediates of its LAST
 * step (any may be NULL).  Layouts: calV, Vm: 6 per body; nu: 1 per
 * suspension; Ym: 3 per body; qm: 4 per body; vb_n, vb_m: 3 per blob. */
typedef struct {
    double* calV;   /* step 2 rigid projection of v-breve at x^n           */
    double* nu;     /* step 3                                               */
    double* Ym;     /* step 4 mid-step centres                              */
    double* qm;     /* step 4 mid-step quaternions                          */
    double* Vm;     /* step 5 mid-step body velocities                      */
    double* vb_n;   /* v-breve at x^n                                       */
    double* vb_m;   /* v-breve at x^m                                       */
    double* FTm;    /* mid-step body forces and torques, 6 per body         */
} gdc_trace;

typedef struct gdc_ctx gdc_ctx;

/* Bytes of device workspace gdc_init needs for these sizes and parameters
 * (0 when an argument is invalid).  tmpl_nblobs: n_templates counts;
 * susp_body_off: n_susp+1 increasing offsets starting at 0; body_tmpl: one
 * template index per body (host arrays). */
size_t gdc_workspace_bytes(const gdc_params* params, int n_templates, const int* tmpl_nblobs,
                           int n_susp, const long long* susp_body_off, const int* body_tmpl);

/* Create a context.  Templates are body-frame blob coordinates (host,
 * 3 doubles per blob, templates back to back); the library re-centres each
 * on its blob centroid, which is then Y_p (Sec. 2).  Y (dev, 3 per body) and
 * q (dev, 4 per body, unit) are the caller's state arrays; gdc_step updates
 * them in place.  Precomputes each template's preconditioner block (FP64
 * Cholesky of its RPY block, Sec. 2.2 and the block-diagonal P described after
 * Eq. lin_sys_RMB) on the device.  stream is a cudaStream_t (NULL = default stream). */
gdc_status gdc_init(gdc_ctx** ctx, const gdc_params* params,
                    int n_templates, const int* tmpl_nblobs, const double* tmpl_xyz,
                    int n_susp, const long long* susp_body_off, const int* body_tmpl,
                    double* Y, double* q, void* workspace, size_t workspace_bytes, void* stream);

void        gdc_destroy(gdc_ctx* ctx);
const char* gdc_last_error(const gdc_ctx* ctx);

/* Change tolerances, precision, divergence mode, scheme, forces or dt of an
 * existing context (sizes and seed are fixed at init). */
gdc_status gdc_set_params(gdc_ctx* ctx, const gdc_params* params);

/* The rigid multiblob mobility problem at the current state (Eq. lin_sys_RMB):
 *   [ M  -K ] [lambda]   [ -vbrev - u_inf ]
 *   [-K^T 0 ] [  V   ] = [ -FT            ]
 * solved by right-preconditioned GMRES with the block-diagonal P (Sec. 2.2).
 * FT (dev, 6 per body), vbrev (dev, 3 per blob, NULL = 0), V (dev out, 6 per
 * body), lambda (dev out, 3 per blob, or NULL).  info (host) may be NULL. */
gdc_status gdc_mobility_solve(gdc_ctx* ctx, const double* FT, const double* vbrev, double* V,
                              double* lambda, gdc_solve_info* info);

/* Advance the state by nsteps steps of the configured scheme (Sec. 3 steps
 * 1-6, or App. D).  Step k draws W and W-tilde from Philox with counter
 * (index, suspension, step, stream).  info: host array of nsteps entries, or NULL. */
gdc_status gdc_step(gdc_ctx* ctx, int nsteps, gdc_step_info* info);
gdc_status gdc_set_trace(gdc_ctx* ctx, const gdc_trace* trace);

/* Checkpoint / resume: copy the state (host arrays, 3 and 4 doubles per body)
 * and the step counter out of / into the context. */
gdc_status gdc_get_state(gdc_ctx* ctx, double* Y_host, double* q_host, unsigned long long* step);
gdc_status gdc_set_state(gdc_ctx* ctx, const double* Y_host, const double* q_host, unsigned long long step);

/* ---- building blocks of the step, exposed for verification -------------- */

/* Blob positions r_i = Y_p + R(q_p) b_i of the current state (dev out, 3 per blob). */
gdc_status gdc_blob_positions(gdc_ctx* ctx, double* r);

/* u = M lambda at the current state (Eq. ddof_mob, RPY of Sec. 4.1); lambda, u dev,
 * 3 per blob; precision is a gdc_precision. */
gdc_status gdc_rpy_apply(gdc_ctx* ctx, int precision, const double* lambda, double* u);

/* The saddle operator [M lambda - K V; -K^T lambda] (Eq. lin_sys_RMB) on x = [lambda; V]
 * stored per suspension as [3 per blob | 6 per body] (dev in, dev out). */
gdc_status gdc_saddle_apply(gdc_ctx* ctx, int precision, const double* x, double* y);

/* z = P^-1 r for the block-diagonal preconditioner (same layout as above). */
gdc_status gdc_precond_apply(gdc_ctx* ctx, const double* r, double* z);

/* vbrev = sqrt(2 kT / dt) M^(1/2) W by Lanczos (Sec. 4.1); W, vbrev dev, 3 per blob. */
gdc_status gdc_brownian_slip(gdc_ctx* ctx, const double* W, double* vbrev, int* iters, double* err);

/* Step 2 (Eq. sol_unconst): calV = (K^T K)^-1 K^T vbrev per body; vbrev dev 3 per blob, calV dev 6 per body. */
gdc_status gdc_lsq_velocity(gdc_ctx* ctx, const double* vbrev, double* calV);

/* Pair forces (gdc_params.potential) between blobs of different bodies, summed per body
 * as [F_p; T_p] (dev out, 6 per body). */
gdc_status gdc_forces(gdc_ctx* ctx, double* FT);

/* The N(0,1) draws of the step counter: stream 0 gives W (3 per blob),
 * stream 1 gives W-tilde (6 per body). */
gdc_status gdc_draw_normals(gdc_ctx* ctx, unsigned long long step, int stream, double* out);

/* Layout helper: offset of each suspension's [lambda; V] block in the
 * vectors of gdc_saddle_apply / gdc_precond_apply (host out, n_susp + 1). */
gdc_status gdc_saddle_offsets(const gdc_ctx* ctx, long long* off);

/* ---- allocation-free RPY product ------------------------------------------
 *
 * For callers that cannot allocate device memory: for example a host program
 * that hands out all device memory from its own fixed pool and forbids any
 * other allocation, or a latency-critical loop that cannot afford the
 * device-wide synchronisation that cudaMalloc / cudaFree may cause.  The
 * paper has no counterpart: this entry point only exists for such callers.
 *
 * u = M lambda for ONE suspension of n_blobs free blobs (no rigid bodies):
 * the unbounded RPY product with the overlapping-blob form, pair terms in
 * FP32 (the library's FP32 pair kernel), chunk sums and the corrections of the
 * self pair and of pairs closer than 2a in FP64.
 * r (dev, 3 doubles per blob, lab positions), lambda (dev, 3 per blob) and
 * u (dev out, 3 per blob) are the caller's; stream is a cudaStream_t.
 *
 * It allocates nothing: its scratch (about 7 MB) is a fixed device array
 * inside the library, present on every GPU that loads the library until the
 * process exits.  The first call on a device looks up that array's device
 * address, so make the first call on each device before any stream capture.
 * n_blobs above GDC_NOALLOC_MAX_BLOBS is rejected with GDC_ERR_INVALID_ARG
 * (message in gdc_last_error(NULL)).  Every call uses the same array: calls
 * that overlap on the GPU (different streams, or different host threads on
 * one device) race and must be serialised by the caller.  The call is
 * asynchronous and returns before the kernels finish, so a failure on the GPU
 * cannot be returned as a status: if a tile copy of the pair kernel does not
 * complete within its bounded wait, every entry of u is set to NaN instead.
 * Each call starts by clearing that flag, so the next call is unaffected. */
#define GDC_NOALLOC_MAX_BLOBS 16384
gdc_status gdc_rpy_apply_noalloc(const double* r, const double* lambda, double* u, int n_blobs,
                                 double a, double eta, void* stream);

/* ---- testing the bounded waits ----------------------------------------------
 *
 * The FP32 pair kernels stage source tiles with bulk copies and wait for each on an
 * mbarrier for at most a bounded number of polls; a wait that gives up makes the kernel
 * wait (again bounded) for its copies in flight and return early, and the call reports
 * GDC_ERR_TIMEOUT (gdc_rpy_apply_noalloc: u set to NaN).  This process-wide setting
 * changes that bound for the pair-kernel launches issued after it (a step graph captured
 * before keeps its bound): polls > 0 sets it, 0 restores the default (400,000 polls), and
 * polls < 0 makes every first wait give up without polling, which exercises the timeout
 * path on purpose.  It is meant for tests of that path, not for production use. */
void gdc_debug_wait_polls(int polls);

/* ---- fluctuating force-coupling method (FCM) in a periodic cube ---------------
 *
 * Sec. 4.2's other way to apply the mobility: M_FCM = J L^-1 S and the Brownian
 * velocities v-breve = J L^-1 D W, on a regular grid of N^3 points in a periodic cube of
 * side L (the implementation Sec. 4.2 and Sec. 6.1 describe):
 *   S  spreads lambda_i with the Gaussian envelope (2 pi sigma^2)^(-3/2) exp(-|x - r_i|^2
 *      / (2 sigma^2)) (Eq. spreading; sigma = a / sqrt(pi) gives the RPY self-mobility),
 *      evaluated at minimum-image distances and cut off beyond R_t (Sec. 6.1: 3a);
 *   L^-1 solves the Stokes equations (Eqs. fluc_stokes1-2) spectrally: mean flow zero, and
 *      every mode with a Nyquist wavenumber component set to zero;
 *   J  averages with the same envelopes by the trapezoidal rule (Eq. averaging, J = S*);
 *   D W is the divergence of the fluctuating stress: six N(0,1) per grid point (Philox
 *      stream 2, counter (k/2, owner, step, 2), normals xx, yy, zz, xy, xz, yz of point
 *      x + N (y + N z)), diagonal entries scaled by 2 sqrt(kT eta / (h^3 dt)) and the others
 *      by sqrt(2 kT eta / (h^3 dt)), h = L/N (Sec. 6.1), so that v-breve has the
 *      covariance (2 kT / dt) M_FCM (Eq. fluctu_dissip in the velocity form of Sec. 3).
 * Grid arithmetic (spreading, FFTs, solve) is FP32; averages are summed in FP32 rows added
 * in FP64.  Positions may lie anywhere (they are wrapped into the cube).
 * All arrays are device arrays of 3 doubles per blob, owned by the caller; calls are
 * asynchronous on the stream given at init and end with a synchronisation.  The context
 * allocates nothing after init: its grids live in the caller's workspace. */
typedef struct gdc_fcm gdc_fcm;

typedef struct {
    int    N;         /* grid points per side: a power of two in [16, 512]          */
    double L;         /* side of the periodic cube                                  */
    double sigma;     /* envelope width                                             */
    double R_t;       /* envelope truncation radius, 0 < R_t < L/2, R_t/(L/N) <= 15  */
    double eta;       /* viscosity                                                  */
    int    max_blobs; /* largest blob count of a call                               */
} gdc_fcm_params;

size_t     gdc_fcm_workspace_bytes(const gdc_fcm_params* params);
gdc_status gdc_fcm_init(gdc_fcm** fcm, const gdc_fcm_params* params, void* workspace, size_t ws_bytes,
                        void* stream);
/* u = M_FCM lambda = J L^-1 S lambda at positions r (n_blobs <= max_blobs). */
gdc_status gdc_fcm_apply(gdc_fcm* fcm, int n_blobs, const double* r, const double* lambda, double* u);
/* Draws the stress of (seed, owner, step), keeps u-breve = L^-1 D W on the grid, and
 * returns v = J u-breve at positions r (kT >= 0, dt > 0). */
gdc_status gdc_fcm_brownian(gdc_fcm* fcm, unsigned long long seed, unsigned int owner, unsigned long long step,
                            double kT, double dt, int n_blobs, const double* r, double* v);
/* v = J u-breve of the last gdc_fcm_brownian at new positions r: the re-averaging that
 * makes changes of configuration cheap for FCM (Sec. 5). */
gdc_status gdc_fcm_average(gdc_fcm* fcm, int n_blobs, const double* r, double* v);
const char* gdc_fcm_last_error(const gdc_fcm* fcm);
unsigned long long gdc_fcm_launches(const gdc_fcm* fcm);   /* kernels launched since init */
void       gdc_fcm_destroy(gdc_fcm* fcm);

/* ---- instrumentation ---------------------------------------------------- */

typedef struct {
    unsigned long long launches;        /* kernels this context launched since gdc_profile */
    unsigned long long rpy32_launches;  /* FP32 RPY pair-kernel launches timed            */
    unsigned long long rpy64_launches;  /* FP64 RPY pair-kernel launches timed            */
    unsigned long long force_launches;  /* repulsion pair-kernel launches timed           */
    double rpy32_ms, rpy64_ms, force_ms; /* summed CUDA-event durations of those launches */
    double pairs_per_product;           /* ordered blob pairs one RPY product evaluates  */
    int    targets_per_thread;          /* pair-kernel tiling in use                     */
    double work_waves;                  /* work items per launch / (4 x SM count)        */
    double autotune_ms;                 /* fastest FP32 product found at init (0: none)  */
    unsigned long long rpydf_launches;  /* double-float residual pair-kernel launches     */
    double rpydf_ms;                    /* their summed CUDA-event durations              */
    int    pair_kernel;                 /* FP32 pair kernel in use: 1 ordered, 2 symmetric */
    int    sym_width;                   /* source tiles per work item (symmetric kernel)  */
    double unique_pairs_per_product;    /* unordered pairs incl. self, sum n (n + 1) / 2  */
    int    min_blocks_per_sm;           /* resident blocks per SM the FP32 pair kernel in use
                                           was compiled for (chosen by the autotuner)     */
    int    df_kernel;                   /* double-float residual kernel in use: 0 ordered,
                                           else the resident blocks per SM (3 or 4) of the
                                           symmetric one (chosen by the autotuner)        */
} gdc_profile_info;

/* FP32 FMA throughput probe (the measured denominator of the pair kernels' FP32 roofline):
 * launches n_blocks blocks of 256 threads on `stream` (a cudaStream_t, NULL = default); each
 * thread runs 8 independent chains of FP32 pairs, x <- x a + b, for `iters` iterations, as
 * scalar FMAs (mode 0), packed fma.rn.f32x2 (mode 1, two FMAs per instruction, as the pair
 * kernels use) or half and half (mode 2), and writes one float to out[block * 256 + thread]
 * (device, n_blocks * 256 floats, caller-owned).  The three modes compute the same values.
 * Work per launch: n_blocks * 256 * iters * 32 flops; the caller times it.
 * GDC_ERR_INVALID_ARG for another mode, n_blocks < 1, iters < 1 or out == NULL;
 * GDC_ERR_CUDA if the launch fails.  Asynchronous; needs no context. */
gdc_status gdc_fma_probe(int mode, int n_blocks, int iters, float* out, void* stream);

/* Reset the counters; enable != 0 also brackets every pair-kernel launch with
 * CUDA events recorded on the context's stream (events are created once). */
gdc_status gdc_profile(gdc_ctx* ctx, int enable);
/* Synchronise the stream and report the counters (host out). */
gdc_status gdc_profile_read(gdc_ctx* ctx, gdc_profile_info* out);

#ifdef __cplusplus
}
#endif
#endif /* GDC_H */
