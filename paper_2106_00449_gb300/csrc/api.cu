// C ABI of the library (include/gdc.h): validation, workspace layout, and the
// orchestration of the gDC step of Sec. 3 (steps 1-6) and the Euler-Maruyama step of
// App. D on top of the kernels of the other translation units.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <new>

#include "common.cuh"
#include "forces.cuh"

namespace gdc {

gdc_status fail(gdc_ctx* c, gdc_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

// the bound of the pair kernels' waits for a tile copy (gdc_debug_wait_polls): 0 = default
static std::atomic<int> g_wait_polls{0};

int first_wait_polls() {
    const int v = g_wait_polls.load();
    return v == 0 ? GDC_WAIT_POLLS : (v < 0 ? 0 : v);
}

gdc_status cuda_check(gdc_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return GDC_OK;
    return fail(c, GDC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---- pair-kernel timing with CUDA events on the library's stream ----

int prof_begin(gdc_ctx* c, int kind) {
    if (!c->prof_on) return -1;
    if (2 * (c->prof_used + 1) > (int)c->prof_ev.size()) prof_flush(c);
    const int idx = c->prof_used++;
    c->prof_kind[idx] = kind;
    cudaEventRecord(c->prof_ev[2 * idx], c->stream);
    return idx;
}

void prof_end(gdc_ctx* c, int idx) {
    if (idx < 0) return;
    cudaEventRecord(c->prof_ev[2 * idx + 1], c->stream);
}

void prof_flush(gdc_ctx* c) {
    if (c->prof_used == 0) return;
    cudaEventSynchronize(c->prof_ev[2 * (c->prof_used - 1) + 1]);
    for (int i = 0; i < c->prof_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]) == cudaSuccess) {
            c->prof_ms[c->prof_kind[i]] += ms;
            c->prof_count[c->prof_kind[i]] += 1;
        }
    }
    c->prof_used = 0;
}

static const char* validate_params(const gdc_params* p) {
    if (!p) return "params is NULL";
    if (!(p->eta > 0.0) || !std::isfinite(p->eta)) return "eta must be > 0";
    if (!(p->kT >= 0.0) || !std::isfinite(p->kT)) return "kT must be >= 0";
    if (!(p->a > 0.0) || !std::isfinite(p->a)) return "a must be > 0";
    if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return "dt must be > 0";
    if (!(p->gmres_tol > 0.0) || !(p->gmres_tol < 1.0)) return "gmres_tol must be in (0, 1)";
    if (p->gmres_max_iter < 1) return "gmres_max_iter must be >= 1";
    if (p->pair_kernel < 0 || p->pair_kernel > 2) return "pair_kernel must be 0 (choose), 1 (ordered) or 2 (symmetric)";
    if (p->gmres_restart < 2 || p->gmres_restart > GDC_MAX_RESTART) return "gmres_restart must be in [2, 100]";
    if (!(p->lanczos_tol > 0.0) || !(p->lanczos_tol < 1.0)) return "lanczos_tol must be in (0, 1)";
    if (p->lanczos_max_iter < 2 || p->lanczos_max_iter > GDC_MAX_LANCZOS) return "lanczos_max_iter must be in [2, 128]";
    if (p->lanczos_precond != 0 && p->lanczos_precond != 1) return "lanczos_precond must be 0 or 1";
    if (p->df_kernel != 0 && p->df_kernel != 1 && p->df_kernel != 3 && p->df_kernel != 4)
        return "df_kernel must be 0 (as pair_kernel), 1 (ordered), 3 or 4 (symmetric, blocks per SM)";
    if (!(p->rfd_delta > 0.0) || !(p->rfd_delta < 1.0)) return "rfd_delta must be in (0, 1)";
    if (p->precision != GDC_FP64 && p->precision != GDC_FP32_MIXED) return "unknown precision";
    if (p->divmode != GDC_DIV_RFD && p->divmode != GDC_DIV_FD) return "unknown divmode";
    if (p->scheme != GDC_SCHEME_GDC && p->scheme != GDC_SCHEME_EM) return "unknown scheme";
    if (!(p->rep_A >= 0.0) || !std::isfinite(p->rep_A)) return "rep_A must be >= 0";
    if (p->rep_A > 0.0 && !(p->rep_b > 0.0)) return "rep_b must be > 0 when rep_A > 0";
    if (!std::isfinite(p->shear_rate)) return "shear_rate must be finite";
    if (p->potential < 0 || p->potential > 2)
        return "potential must be 0 (soft sphere), 1 (repel-attract) or 2 (repel-attract-repel)";
    if (!(p->well_A >= 0.0) || !std::isfinite(p->well_A)) return "well_A must be >= 0";
    if (p->potential > 0 && p->well_A > 0.0 && !(p->well_lambda > 0.0 && std::isfinite(p->well_lambda)))
        return "well_lambda must be > 0 when the wells are on";
    if (p->force_method < 0 || p->force_method > 2)
        return "force_method must be 0 (choose), 1 (all pairs) or 2 (cell list)";
    if (p->mobility != GDC_MOB_RPY && p->mobility != GDC_MOB_FCM) return "mobility must be 0 (RPY) or 1 (FCM)";
    if (p->mobility == GDC_MOB_FCM) {
        const gdc_fcm_params fp = fcm_params_of(*p, 1);
        if (gdc_fcm_workspace_bytes(&fp) == 0)
            return "FCM needs box_L > 0 and a valid grid: fcm_N a power of two in [16, 512], 0 < R_t < box_L/2, "
                   "R_t within 15 grid spacings";
        if (forces_on(*p) && std::floor(p->box_L / (force_cutoff(*p) * (1.0 + 1e-4))) < 3.0)
            return "with the periodic FCM mobility the pair-force cutoff must fit 3 times in box_L";
        if (p->shear_rate != 0.0) return "a background shear is not periodic: not available with the FCM mobility";
    }
    if (p->wall != 0 && p->wall != 1) return "wall must be 0 or 1";
    if (p->wall) {
        if (p->mobility != GDC_MOB_RPY) return "the wall-corrected mobility is an RPY mobility (mobility 0)";
        if (p->shear_rate != 0.0) return "a background shear is not available above a wall";
        if (!(p->wall_V0 >= 0.0) || !std::isfinite(p->wall_V0)) return "wall_V0 must be >= 0";
        if (p->wall_V0 > 0.0 && !(p->wall_b > 0.0 && std::isfinite(p->wall_b))) return "wall_b must be > 0";
        if (!std::isfinite(p->body_weight)) return "body_weight must be finite";
    } else if (p->wall_V0 != 0.0 || p->body_weight != 0.0) {
        return "wall_V0 and body_weight need wall = 1";
    }
    return nullptr;
}

// Host-side layout of a context from the user's sizes (no device work).
static const char* build_host_layout(gdc_ctx* c, const gdc_params* p, int n_templates, const int* tmpl_nblobs,
                                     int n_susp, const long long* susp_body_off, const int* body_tmpl) {
    if (const char* m = validate_params(p)) return m;
    if (n_templates < 1 || !tmpl_nblobs) return "need at least one template";
    if (n_susp < 1 || !susp_body_off) return "need at least one suspension";
    if (susp_body_off[0] != 0) return "susp_body_off[0] must be 0";
    if (p->mobility == GDC_MOB_FCM && n_susp != 1) return "the FCM mobility takes one suspension";
    for (int s = 0; s < n_susp; ++s)
        if (susp_body_off[s + 1] < susp_body_off[s]) return "susp_body_off must be non-decreasing";
    const long long NB = susp_body_off[n_susp];
    if (NB < 1) return "no bodies";
    if (NB > (1LL << 24)) return "too many bodies (at most 2^24)";
    if (!body_tmpl) return "body_tmpl is NULL";
    c->p = *p;
    c->T = n_templates;
    c->S = n_susp;
    c->NB = (int)NB;
    c->h_tmpl_n.assign(tmpl_nblobs, tmpl_nblobs + n_templates);
    c->h_tmpl_off.assign(n_templates + 1, 0);
    c->h_minv_off.assign(n_templates + 1, 0);
    for (int t = 0; t < n_templates; ++t) {
        if (tmpl_nblobs[t] < 1 || tmpl_nblobs[t] > GDC_MAX_TMPL_BLOBS) return "template blob count must be in [1, 340]";
        c->h_tmpl_off[t + 1] = c->h_tmpl_off[t] + tmpl_nblobs[t];
        c->h_minv_off[t + 1] = c->h_minv_off[t] + 9LL * tmpl_nblobs[t] * tmpl_nblobs[t];
    }
    c->h_body_off.assign(susp_body_off, susp_body_off + n_susp + 1);
    c->h_body_tmpl.assign(body_tmpl, body_tmpl + NB);
    c->h_body_blob_off.assign(NB + 1, 0);
    c->h_body_susp.assign(NB, 0);
    c->max_body_blobs = 0;
    for (long long b = 0; b < NB; ++b) {
        const int t = body_tmpl[b];
        if (t < 0 || t >= n_templates) return "body_tmpl entry out of range";
        c->h_body_blob_off[b + 1] = c->h_body_blob_off[b] + tmpl_nblobs[t];
        c->max_body_blobs = std::max(c->max_body_blobs, tmpl_nblobs[t]);
    }
    const long long NBL = c->h_body_blob_off[NB];
    if (3 * NBL + 6 * NB > (1LL << 30)) return "too many blobs";
    c->NBL = (int)NBL;
    c->h_blob_off.assign(n_susp + 1, 0);
    c->h_gm_off.assign(n_susp + 1, 0);
    for (int s = 0; s < n_susp; ++s) {
        for (long long b = susp_body_off[s]; b < susp_body_off[s + 1]; ++b) c->h_body_susp[b] = s;
        c->h_blob_off[s + 1] = c->h_body_blob_off[susp_body_off[s + 1]];
        const long long nbl = c->h_blob_off[s + 1] - c->h_blob_off[s];
        const long long nbd = susp_body_off[s + 1] - susp_body_off[s];
        c->h_gm_off[s + 1] = c->h_gm_off[s] + 3 * nbl + 6 * nbd;
    }
    c->ngm = c->h_gm_off[n_susp];
    c->m = p->gmres_restart;
    c->kmax = p->lanczos_max_iter;
    c->red_cols = std::max(c->m + 1, c->kmax + 1);
    c->red_cols = (c->red_cols + 7) / 8 * 8;
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    c->device = dev;
    c->num_sms = sms;
    // bodies per block of the factor products: as many as keep 8 blocks per SM busy (at most
    // GDC_TB_MAX), fewer for large templates (at most 2,048 rows per block: 40 KB of shared
    // memory in the factor products, 41 KB in the preconditioner); below 4 per
    // block the products keep one block per body (measured faster there: 2,520 bodies)
    {
        int B = 1;
        while (B < GDC_TB_MAX && NB >= 2LL * B * 8 * sms) B *= 2;
        c->tb_use = B >= 4;
        c->lz_qbuf_on = n_susp > sms;   // the eigen-step's scratch: see krylov.cu
        std::vector<std::vector<int>> by_t(n_templates);
        for (long long b = 0; b < NB; ++b) by_t[body_tmpl[b]].push_back((int)b);
        c->h_tb_items.clear();
        c->h_tb_bodies.clear();
        c->tb_smem = 0;
        c->tb_precond_smem = 0;
        for (int t = 0; t < n_templates; ++t) {
            const int n3 = 3 * tmpl_nblobs[t];
            const int bt = std::max(1, std::min(B, 2048 / n3));
            for (size_t i = 0; i < by_t[t].size(); i += bt) {
                const int cnt = (int)std::min<size_t>(bt, by_t[t].size() - i);
                c->h_tb_items.push_back(make_int4(t, (int)c->h_tb_bodies.size() + (int)i, cnt, 0));
                c->tb_smem = std::max(c->tb_smem, (size_t)cnt * n3 * 2 * sizeof(double));
                c->tb_precond_smem = std::max(c->tb_precond_smem,
                                              (size_t)cnt * ((2 * n3 + 16) * sizeof(double) + n3 * sizeof(float)));
            }
            c->h_tb_bodies.insert(c->h_tb_bodies.end(), by_t[t].begin(), by_t[t].end());
        }
        c->tb_n_items = (int)c->h_tb_items.size();
    }
    plan_mv_capacity(c);
    setup_segments(c);
    c->h_blk_off.assign(NB + 1, 0);
    for (long long b = 0; b < NB; ++b) {
        const long long n3 = 3 * (c->h_body_blob_off[b + 1] - c->h_body_blob_off[b]);
        c->h_blk_off[b + 1] = c->h_blk_off[b] + (p->wall ? n3 * n3 : 0);
    }
    if (p->wall) build_wall_items(c);
    return nullptr;
}

// Sequential carving of the caller's workspace with 256-byte alignment.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base((char*)b) {}
    template <typename T>
    T* take(long long count) {
        off = (off + 255) & ~(size_t)255;
        T* ptr = base ? (T*)(base + off) : nullptr;
        off += sizeof(T) * (size_t)std::max<long long>(count, 1);
        return ptr;
    }
};

static size_t carve(gdc_ctx* c, void* base) {
    Carver w(base);
    const long long S = c->S, NB = c->NB, NBL = c->NBL, T = c->T;
    const long long nt = c->h_tmpl_off[T];
    const long long cols = c->red_cols;
    c->susp_body_off = w.take<long long>(S + 1);
    c->susp_blob_off = w.take<long long>(S + 1);
    c->susp_gm_off = w.take<long long>(S + 1);
    c->body_blob_off = w.take<long long>(NB + 1);
    c->minv_off = w.take<long long>(T + 1);
    c->body_tmpl = w.take<int>(NB);
    c->tb_items = w.take<int4>(NB);
    c->tb_bodies = w.take<int>(NB);
    c->body_susp = w.take<int>(NB);
    c->blob_body = w.take<int>(NBL);
    c->blob_susp = w.take<int>(NBL);
    c->tmpl_n = w.take<int>(T);
    c->tmpl_off = w.take<int>(T + 1);
    c->blob_gm = w.take<int>(NBL);
    c->body_gm = w.take<int>(NB);
    c->tmpl_xyz = w.take<double>(3 * nt);
    c->tmpl_L = w.take<double>(T);
    c->tmpl_Minv = w.take<double>(c->h_minv_off[T]);
    c->tmpl_M = w.take<double>(c->h_minv_off[T]);
    c->tmpl_M32 = w.take<float>(c->h_minv_off[T]);
    c->tmpl_Minv32 = w.take<float>(c->h_minv_off[T]);
    c->tmpl_G = w.take<double>(18 * nt);
    c->tmpl_N = w.take<double>(36 * T);
    c->tmpl_KtKp = w.take<double>(36 * T);
    c->tmpl_work = w.take<double>(2 * c->h_minv_off[T]);
    c->tmpl_LT = w.take<double>(c->h_minv_off[T]);
    c->tmpl_X = w.take<double>(c->h_minv_off[T]);
    c->tmpl_XT = w.take<double>(c->h_minv_off[T]);
    c->tmpl_X32 = w.take<float>(c->h_minv_off[T]);
    c->tmpl_XT32 = w.take<float>(c->h_minv_off[T]);
    c->body_L = w.take<double>(NB);
    c->Rb = w.take<double>(9 * NB);
    c->r = w.take<double>(3 * NBL);
    c->Yc = w.take<double>(3 * NB);
    c->ref = w.take<double>(3 * S);
    c->spos = w.take<float4>(NBL);
    c->slam = w.take<float4>(NBL);
    c->sdup = w.take<float4>(3 * NBL);
    c->spos64 = w.take<double4_32a>(NBL);
    c->slam64 = w.take<double4_32a>(NBL);
    c->W = w.take<double>(3 * NBL);
    c->Wt = w.take<double>(6 * NB);
    c->vb_n = w.take<double>(3 * NBL);
    c->vb_t = w.take<double>(3 * NBL);
    c->vb_m = w.take<double>(3 * NBL);
    c->calV = w.take<double>(6 * NB);
    c->calVt = w.take<double>(6 * NB);
    c->Yt = w.take<double>(3 * NB);
    c->qt = w.take<double>(4 * NB);
    c->Ym = w.take<double>(3 * NB);
    c->qm = w.take<double>(4 * NB);
    c->FT = w.take<double>(6 * NB);
    c->Vm = w.take<double>(6 * NB);
    c->nu = w.take<double>(S);
    c->divp = w.take<double>(S);
    c->fblob = w.take<double>(3 * NBL);
    if (c->p.mobility == GDC_MOB_FCM) {
        const gdc_fcm_params fp = fcm_params_of(c->p, NBL);
        c->fcm_ws_bytes = gdc_fcm_workspace_bytes(&fp);
        c->fcm_u = w.take<double>(3 * NBL);
        c->fcm_Mt = w.take<double>(c->h_minv_off[T]);
        c->fcm_ws = (void*)w.take<char>((long long)c->fcm_ws_bytes);
    }
    c->cell_H = cell_buckets(NBL);
    c->cell_xyz = w.take<int4>(NBL);
    c->cell_key = w.take<unsigned>(NBL);
    c->cell_cnt = w.take<int>(c->cell_H);
    c->cell_start = w.take<int>(c->cell_H);
    c->cell_fill = w.take<int>(c->cell_H);
    c->cell_list = w.take<int>(NBL);
    c->cell_scan = w.take<int>(cell_scan_ints(NBL));
    c->u3 = w.take<double>(3 * NBL);
    const long long m = c->m, n = c->ngm;
    c->gm_V = w.take<double>((m + 1) * n);
    c->gm_x = w.take<double>(n);
    c->gm_b = w.take<double>(n);
    c->gm_r = w.take<double>(n);
    c->gm_w = w.take<double>(n);
    c->gm_z = w.take<double>(n);
    c->gm_H = w.take<double>(S * (m + 1) * m);
    c->gm_cs = w.take<double>(S * m);
    c->gm_sn = w.take<double>(S * m);
    c->gm_g = w.take<double>(S * (m + 1));
    c->gm_y = w.take<double>(S * cols);
    c->gm_h = w.take<double>(S * cols);
    c->gm_h2 = w.take<double>(S * cols);
    c->gm_bnorm = w.take<double>(S);
    c->gm_res = w.take<double>(2 * S);
    c->gm_scal = w.take<double>(S);
    c->gm_active = w.take<int>(2 * S);
    c->gm_j = w.take<int>(S);
    const long long k = c->kmax, nl = 3 * NBL;
    c->lz_V = w.take<double>((k + 1) * nl);
    c->lz_w = w.take<double>(nl);
    c->lz_alpha = w.take<double>(S * k);
    c->lz_beta = w.take<double>(S * k);
    c->lz_c = w.take<double>(S * k);
    c->lz_lastk = w.take<int>(2 * S);
    c->lz_hint = w.take<int>(S);
    c->lz_qbuf = w.take<double>(c->lz_qbuf_on ? (long long)S * lz_q_doubles(c->kmax) : 1);
    c->lz_h = w.take<double>(S * cols);
    c->lz_Wnorm = w.take<double>(S);
    c->lz_err = w.take<double>(S);
    c->lz_scal = w.take<double>(S);
    c->lz_active = w.take<int>(S);
    c->lz_k = w.take<int>(S);
    c->lz_fix = w.take<int>(S);
    c->lz_z = w.take<double>(nl);
    c->lz_u = w.take<double>(nl);
    c->seg_gm.chunks = w.take<Chunk>(c->seg_gm.n_chunks);
    c->seg_gm.seg_chunk_off = w.take<int>(S + 1);
    c->seg_gm.off = c->susp_gm_off;
    c->seg_lz.chunks = w.take<Chunk>(c->seg_lz.n_chunks);
    c->seg_lz.seg_chunk_off = w.take<int>(S + 1);
    c->red_part = w.take<double>((long long)std::max(c->seg_gm.n_chunks, c->seg_lz.n_chunks) * cols);
    c->mv_items = w.take<MvItem>(c->mv_cap_items);
    c->mv_nk = w.take<int>(S);
    c->mv_part = (void*)w.take<double4_32a>((long long)c->mv_cap_kmax * NBL);
    c->dev_status = w.take<int>(4);
    c->sym_items = w.take<SymItem>(c->sym_cap_items);
    c->sym_row_nk = w.take<int>(std::max<long long>(1, c->sym_n_tiles));
    c->sym_tile_base = w.take<long long>(S + 1);
    c->sym_jbase = w.take<long long>(S + 1);
    c->sym_part_i = w.take<float4>((long long)c->sym_cap_kmax * NBL);
    c->sym_part_j = w.take<float4>(std::max<long long>(1, c->sym_n_jslots) * GDC_SYM_TILE);
    c->dfs_items = w.take<SymItem>(c->dfs_n_items);
    c->dfs_row_nk = w.take<int>(std::max<long long>(1, c->sym_n_tiles));
    c->dfs_part_i = w.take<double4_32a>((long long)c->dfs_kmax * NBL);
    c->dfs_part_j = w.take<double4_32a>(std::max<long long>(1, c->sym_n_jslots) * GDC_SYM_TILE);
    c->h_near_items.clear();
    for (int s = 0; s < c->S; ++s) {
        const long long ns = c->h_blob_off[s + 1] - c->h_blob_off[s];
        for (long long t0 = 0; t0 < ns; t0 += 256)
            for (long long j0 = 0; j0 < ns; j0 += GDC_NEAR_SRC)
                c->h_near_items.push_back(make_int4(s, (int)t0, (int)j0, (int)std::min(ns, j0 + GDC_NEAR_SRC)));
    }
    c->n_near_items = (int)c->h_near_items.size();
    c->near_items = w.take<int4>(c->n_near_items);
    c->near_cnt = w.take<int>(NBL);
    c->near_idx = w.take<int>((long long)GDC_NEAR_CAP * NBL);
    c->ctl = w.take<LoopCtl>(1);
    c->rep = w.take<StepReport>(1);
    c->lz_vcur = w.take<double>(nl);
    c->gm_vcur = w.take<double>(n);
    if (c->p.wall) {
        const long long tot = c->h_blk_off[NB];
        c->blk_off = w.take<long long>(NB + 1);
        c->blk_work = w.take<double>(2 * tot);
        c->blk_Minv = w.take<double>(tot);
        c->blk_LT = w.take<double>(tot);
        c->blk_X = w.take<double>(tot);
        c->blk_XT = w.take<double>(tot);
        c->blk_G = w.take<double>(18 * NBL);
        c->blk_N = w.take<double>(36 * NB);
        c->wall_items = w.take<int2>((long long)c->h_wall_items.size());
    }
    return w.off + 256;
}

template <typename T>
static cudaError_t up(gdc_ctx* c, T* dst, const T* src, size_t count) {
    return cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, c->stream);
}

static gdc_status upload_layout(gdc_ctx* c, const double* tmpl_xyz_centred) {
    const int S = c->S, NB = c->NB, NBL = c->NBL, T = c->T;
    std::vector<int> blob_body(NBL), blob_susp(NBL), blob_gm(NBL), body_gm(NB);
    std::vector<double> body_L(NB);
    for (int b = 0; b < NB; ++b) {
        const int s = c->h_body_susp[b];
        const long long lb = b - c->h_body_off[s];
        body_gm[b] = (int)(c->h_gm_off[s] + 3 * (c->h_blob_off[s + 1] - c->h_blob_off[s]) + 6 * lb);
        body_L[b] = c->h_tmpl_L[c->h_body_tmpl[b]];
        for (long long i = c->h_body_blob_off[b]; i < c->h_body_blob_off[b + 1]; ++i) {
            blob_body[i] = b;
            blob_susp[i] = s;
            blob_gm[i] = (int)(c->h_gm_off[s] + 3 * (i - c->h_blob_off[s]));
        }
    }
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(up(c, c->susp_body_off, c->h_body_off.data(), S + 1));
    chk(up(c, c->susp_blob_off, c->h_blob_off.data(), S + 1));
    chk(up(c, c->susp_gm_off, c->h_gm_off.data(), S + 1));
    chk(up(c, c->body_blob_off, c->h_body_blob_off.data(), NB + 1));
    chk(up(c, c->minv_off, c->h_minv_off.data(), T + 1));
    chk(up(c, c->body_tmpl, c->h_body_tmpl.data(), NB));
    chk(up(c, c->tb_items, c->h_tb_items.data(), c->h_tb_items.size()));
    chk(up(c, c->tb_bodies, c->h_tb_bodies.data(), c->h_tb_bodies.size()));
    chk(up(c, c->body_susp, c->h_body_susp.data(), NB));
    chk(up(c, c->blob_body, blob_body.data(), NBL));
    chk(up(c, c->blob_susp, blob_susp.data(), NBL));
    chk(up(c, c->tmpl_n, c->h_tmpl_n.data(), T));
    chk(up(c, c->tmpl_off, c->h_tmpl_off.data(), T + 1));
    chk(up(c, c->blob_gm, blob_gm.data(), NBL));
    chk(up(c, c->body_gm, body_gm.data(), NB));
    chk(up(c, c->tmpl_xyz, tmpl_xyz_centred, 3 * c->h_tmpl_off[T]));
    chk(up(c, c->tmpl_L, c->h_tmpl_L.data(), T));
    chk(up(c, c->body_L, body_L.data(), NB));
    chk(up(c, c->seg_gm.chunks, c->seg_gm.h_chunks.data(), c->seg_gm.h_chunks.size()));
    chk(up(c, c->seg_gm.seg_chunk_off, c->seg_gm.h_seg_chunk_off.data(), S + 1));
    chk(up(c, c->seg_lz.chunks, c->seg_lz.h_chunks.data(), c->seg_lz.h_chunks.size()));
    chk(up(c, c->seg_lz.seg_chunk_off, c->seg_lz.h_seg_chunk_off.data(), S + 1));
    chk(up(c, c->mv_items, c->h_mv_items.data(), c->h_mv_items.size()));
    chk(up(c, c->near_items, c->h_near_items.data(), c->h_near_items.size()));
    chk(up(c, c->mv_nk, c->h_mv_nk.data(), S));
    chk(up(c, c->dfs_items, c->h_dfs_items.data(), c->h_dfs_items.size()));
    chk(up(c, c->dfs_row_nk, c->h_dfs_row_nk.data(), c->h_dfs_row_nk.size()));
    if (c->p.wall) {
        chk(up(c, c->blk_off, c->h_blk_off.data(), NB + 1));
        chk(up(c, c->wall_items, c->h_wall_items.data(), c->h_wall_items.size()));
    }
    chk(cudaMemsetAsync(c->dev_status, 0, 4 * sizeof(int), c->stream));
    chk(cudaMemsetAsync(c->lz_hint, 0, sizeof(int) * S, c->stream));
    chk(cudaStreamSynchronize(c->stream));  // host vectors above go out of scope
    return cuda_check(c, e, "upload of the layout");
}

static gdc_status check_state_host(gdc_ctx* c, const double* Y, const double* q) {
    for (int p = 0; p < c->NB; ++p) {
        double n2 = 0.0;
        for (int k = 0; k < 4; ++k) n2 += q[4 * p + k] * q[4 * p + k];
        if (!(std::fabs(n2 - 1.0) <= 1e-10)) return fail(c, GDC_ERR_INVALID_ARG, "quaternion of body " + std::to_string(p) + " is not unit");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(Y[3 * p + k])) return fail(c, GDC_ERR_INVALID_ARG, "non-finite body centre");
    }
    return GDC_OK;
}

// Clears the device status words once a failure they flagged has been reported, so that the
// next call of the context starts clean.
static gdc_status clear_status(gdc_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->dev_status, 0, 4 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_check(c, e, "status reset");
}

static gdc_status read_status(gdc_ctx* c) {
    int st[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(st, c->dev_status, sizeof(st), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "status read");
    if ((st[0] != 0 || st[1] != 0 || st[2] != 0) && clear_status(c) != GDC_OK) return GDC_ERR_CUDA;
    // a timed-out tile copy first: an incomplete product explains any later failure
    if (st[1] != 0) return fail(c, GDC_ERR_TIMEOUT, "a pair-kernel tile copy did not complete in time");
    if (st[2] != 0) return fail(c, GDC_ERR_NONFINITE, "a blob centre reached the wall (height <= a)");
    if (st[0] == 1) return fail(c, GDC_ERR_NONFINITE, "template RPY block is not positive definite");
    if (st[0] == 2) return fail(c, GDC_ERR_NOT_CONVERGED, "tridiagonal eigensolver did not converge");
    return GDC_OK;
}

// The outcome of a call that failed on the host side: a failure the kernels flagged in the
// status words (a timed-out tile copy, a failed eigen-step) is the cause of the later
// symptom (a Krylov loop that did not converge on an incomplete product), so it takes
// precedence.  The words are cleared once read.
static gdc_status settle(gdc_ctx* c, gdc_status st) {
    if (st == GDC_ERR_CUDA) return st;   // the stream may not be usable
    const gdc_status s2 = read_status(c);
    return s2 != GDC_OK ? s2 : st;
}

// FCM mode: each template's block of M_FCM for the template alone at the centre of the
// periodic cube (3 n_t FCM products on unit vectors), symmetrised (J = S*).  It replaces the
// RPY template block in the block-diagonal preconditioner; R M_t R^T matches a body's block
// up to the small anisotropy of its periodic images.
static gdc_status fcm_template_blocks(gdc_ctx* c) {
    std::vector<double> M(c->h_minv_off[c->T]);
    for (int t = 0; t < c->T; ++t) {
        const int n = c->h_tmpl_n[t], n3 = 3 * n;
        std::vector<double> r(n3), e(n3, 0.0), u(n3);
        for (int i = 0; i < n3; ++i) r[i] = 0.5 * c->p.box_L + c->h_tmpl_xyz[3LL * c->h_tmpl_off[t] + i];
        cudaError_t ce = cudaMemcpyAsync(c->vb_n, r.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, c->stream);
        if (ce != cudaSuccess) return cuda_check(c, ce, "FCM template blocks");
        double* Mb = M.data() + c->h_minv_off[t];
        for (int k = 0; k < n3; ++k) {
            e[k] = 1.0;
            ce = cudaMemcpyAsync(c->W, e.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, c->stream);
            e[k] = 0.0;
            if (ce != cudaSuccess) return cuda_check(c, ce, "FCM template blocks");
            const gdc_status st = gdc_fcm_apply(c->fcm, n, c->vb_n, c->W, c->vb_t);
            if (st != GDC_OK) return fail(c, st, std::string("FCM: ") + gdc_fcm_last_error(c->fcm));
            ce = cudaMemcpyAsync(u.data(), c->vb_t, sizeof(double) * n3, cudaMemcpyDeviceToHost, c->stream);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
            if (ce != cudaSuccess) return cuda_check(c, ce, "FCM template blocks");
            for (int row = 0; row < n3; ++row) Mb[(long long)row * n3 + k] = u[row];
        }
        for (int i = 0; i < n3; ++i)
            for (int j = i + 1; j < n3; ++j) {
                const double m = 0.5 * (Mb[(long long)i * n3 + j] + Mb[(long long)j * n3 + i]);
                Mb[(long long)i * n3 + j] = Mb[(long long)j * n3 + i] = m;
            }
    }
    return cuda_check(c, cudaMemcpyAsync(c->fcm_Mt, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice,
                                         c->stream), "FCM template blocks");
}

// ---- the steps -------------------------------------------------------------------------

static void load_at(gdc_ctx* c, const double* Y, const double* q) {
    launch_ref(c, Y);
    load_config(c, Y, q);
}

static gdc_status forces_at_loaded(gdc_ctx* c, double* FT) {
    if (forces_on(c->p) || c->p.wall) {
        if (forces_on(c->p))
            launch_forces(c, c->p.precision, c->fblob);
        else
            cudaMemsetAsync(c->fblob, 0, sizeof(double) * 3 * c->NBL, c->stream);
        if (c->p.wall) launch_wall_forces(c, c->fblob);   // Sec. 6.2: wall repulsion and weight
        launch_body_KT(c, c->fblob, 0, FT, 0, 1.0);
    } else {
        cudaMemsetAsync(FT, 0, sizeof(double) * 6 * c->NB, c->stream);
    }
    return GDC_OK;
}

// v-breve = sqrt(2 kT / dt) M^(1/2) W at the loaded configuration.  FCM: the step's
// fluctuating field is drawn at the step's first slip and averaged again at later ones.
static gdc_status slip_at_loaded(gdc_ctx* c, const double* W, double* vb, int fixed, int* iters, double* err) {
    const double scale = std::sqrt(2.0 * c->p.kT / c->p.dt);
    if (c->p.kT == 0.0) {
        if (iters) *iters = 0;
        if (err) *err = 0.0;
        return cuda_check(c, cudaMemsetAsync(vb, 0, sizeof(double) * 3 * c->NBL, c->stream), "memset");
    }
    if (c->fcm) {
        if (iters) *iters = 0;
        if (err) *err = 0.0;
        gdc_status st;
        if (c->fcm_field_step != c->step) {
            st = gdc_fcm_brownian(c->fcm, c->p.seed, 0u, c->step, c->p.kT, c->p.dt, (int)c->NBL, c->r, vb);
            if (st == GDC_OK) c->fcm_field_step = c->step;
        } else {
            st = gdc_fcm_average(c->fcm, (int)c->NBL, c->r, vb);
        }
        return st == GDC_OK ? st : fail(c, st, std::string("FCM: ") + gdc_fcm_last_error(c->fcm));
    }
    return lanczos_sqrt(c, W, vb, scale, fixed, iters, err);
}

static gdc_status one_step(gdc_ctx* c, gdc_step_info* info) {
    gdc_step_info inf{};
    inf.step = c->step;
    gdc_status st;
    const double dt = c->p.dt;
    int matvecs = 0;
    launch_normals(c, c->step, 0, c->W);
    launch_normals(c, c->step, 1, c->Wt);
    if (c->p.scheme == GDC_SCHEME_EM) {
        // App. D: one full solve at x^n, then x^(n+1) = x^n + dt V^n
        load_at(c, c->Y, c->q);
        forces_at_loaded(c, c->FT);
        if ((st = slip_at_loaded(c, c->W, c->vb_m, 0, &inf.lanczos_iters[2], &inf.lanczos_err)) != GDC_OK) return st;
        launch_rhs(c, c->vb_m, c->FT, c->gm_b);
        st = gmres_solve(c, c->gm_b, c->gm_x, &inf.solve);
        if (st != GDC_OK) return st;
        launch_scatter_solution(c, c->gm_x, c->Vm, nullptr);
        if ((st = read_status(c)) != GDC_OK) return st;   // no advance on a flagged failure
        launch_advance(c, c->Y, c->q, c->Vm, dt, nullptr, c->Y, c->q);
        matvecs = inf.lanczos_iters[2] + inf.solve.matvecs_fp32 + inf.solve.matvecs_fp64;
    } else {
        // step 2 at x^n
        load_at(c, c->Y, c->q);
        if ((st = slip_at_loaded(c, c->W, c->vb_n, 0, &inf.lanczos_iters[0], &inf.lanczos_err)) != GDC_OK) return st;
        launch_lsq(c, c->vb_n, c->calV);
        // step 3: divergence of calV
        double e2 = 0.0;
        if (c->p.divmode == GDC_DIV_RFD) {
            launch_perturb(c, c->Y, c->q, c->Wt, c->p.rfd_delta, c->Yt, c->qt);
            load_config(c, c->Yt, c->qt);  // same reference point as x^n
            cudaMemcpyAsync(c->lz_fix, c->lz_k, sizeof(int) * c->S, cudaMemcpyDeviceToDevice, c->stream);
            if ((st = slip_at_loaded(c, c->W, c->vb_t, 1, &inf.lanczos_iters[1], &e2)) != GDC_OK) return st;
            launch_lsq(c, c->vb_t, c->calVt);
            launch_rfd_div(c, c->Wt, c->calV, c->calVt, c->p.rfd_delta, dt, c->nu);
        } else {
            int maxn = 0;
            for (int s = 0; s < c->S; ++s) maxn = std::max<int>(maxn, (int)(c->h_body_off[s + 1] - c->h_body_off[s]));
            cudaMemcpyAsync(c->lz_fix, c->lz_k, sizeof(int) * c->S, cudaMemcpyDeviceToDevice, c->stream);
            for (int pl = 0; pl < maxn; ++pl)
                for (int coord = 0; coord < 6; ++coord) {
                    launch_perturb_one(c, c->Y, c->q, pl, coord, c->p.rfd_delta, c->Yt, c->qt);
                    load_config(c, c->Yt, c->qt);
                    int it = 0;
                    if ((st = slip_at_loaded(c, c->W, c->vb_t, 1, &it, &e2)) != GDC_OK) return st;
                    inf.lanczos_iters[1] += it;
                    launch_lsq(c, c->vb_t, c->calVt);
                    launch_fd_accum(c, c->calV, c->calVt, pl, coord, c->p.rfd_delta, c->divp, pl == 0 && coord == 0);
                }
            launch_nu_from_div(c, c->divp, dt, c->nu);
        }
        // step 4: mid-step
        launch_advance(c, c->Y, c->q, c->calV, 0.5 * dt, nullptr, c->Ym, c->qm);
        // step 5: forces and the full mobility solve at the mid-step, same W
        load_at(c, c->Ym, c->qm);
        forces_at_loaded(c, c->FT);
        double e3 = 0.0;
        if ((st = slip_at_loaded(c, c->W, c->vb_m, 0, &inf.lanczos_iters[2], &e3)) != GDC_OK) return st;
        inf.lanczos_err = std::max(inf.lanczos_err, e3);
        launch_rhs(c, c->vb_m, c->FT, c->gm_b);
        st = gmres_solve(c, c->gm_b, c->gm_x, &inf.solve);
        if (st != GDC_OK) return st;
        launch_scatter_solution(c, c->gm_x, c->Vm, nullptr);
        if ((st = read_status(c)) != GDC_OK) return st;   // no advance on a flagged failure
        // step 6
        launch_advance(c, c->Y, c->q, c->Vm, dt, c->nu, c->Y, c->q);
        matvecs = inf.lanczos_iters[0] + inf.lanczos_iters[1] + inf.lanczos_iters[2] + inf.solve.matvecs_fp32 +
                  inf.solve.matvecs_fp64;
    }
    // nu range and a finiteness check
    std::vector<double> nu(c->S, 1.0);
    if (c->p.scheme == GDC_SCHEME_GDC) {
        cudaError_t e = cudaMemcpyAsync(nu.data(), c->nu, sizeof(double) * c->S, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if ((st = cuda_check(c, e, "nu read")) != GDC_OK) return st;
    }
    inf.nu_min = *std::min_element(nu.begin(), nu.end());
    inf.nu_max = *std::max_element(nu.begin(), nu.end());
    if (!std::isfinite(inf.nu_min) || !std::isfinite(inf.nu_max)) return fail(c, GDC_ERR_NONFINITE, "non-finite nu");
    inf.pair_evals = (double)matvecs * c->pair_evals_per_matvec;
    if (c->have_trace) {
        const gdc_trace& t = c->trace;
        auto cp = [&](double* dst, const double* src, long long n) {
            if (dst) cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream);
        };
        cp(t.calV, c->calV, 6LL * c->NB);
        cp(t.nu, c->nu, c->S);
        cp(t.Ym, c->Ym, 3LL * c->NB);
        cp(t.qm, c->qm, 4LL * c->NB);
        cp(t.Vm, c->Vm, 6LL * c->NB);
        cp(t.vb_n, c->vb_n, 3LL * c->NBL);
        cp(t.vb_m, c->vb_m, 3LL * c->NBL);
        cp(t.FTm, c->FT, 6LL * c->NB);
    }
    c->step++;
    if ((st = read_status(c)) != GDC_OK) return st;
    if (info) *info = inf;
    return cuda_check(c, cudaGetLastError(), "step launch");
}

// ---- graph mode: one CUDA graph per step ----------------------------------------------
//
// The whole step (Sec. 3 steps 1-6, or App. D) is captured once as a CUDA graph; the
// Lanczos and GMRES loops inside it are WHILE nodes whose conditions the loop kernels set
// on the device.  A replay needs one device-to-host read (the StepReport) at its end.
// Values the captured launches take by value (tolerances, dt, the trace pointers) are
// fixed at capture: gdc_set_params and gdc_set_trace drop the graph.  Profiling with
// CUDA events around launches, and the FD divergence, use the host-driven path.

__global__ void k_step_begin(StepReport* rep) {
    int* w = reinterpret_cast<int*>(rep);
    for (int i = threadIdx.x; i < (int)(sizeof(StepReport) / sizeof(int)); i += blockDim.x) w[i] = 0;
}

// the state is advanced only when no stage failed (the host-driven path returns early instead)
__global__ void k_step_ok(StepReport* rep, const int* __restrict__ status) {
    const bool bad = rep->lz_notconv[0] || rep->lz_notconv[1] || rep->lz_notconv[2] || rep->gm_bad ||
                     rep->gm_notconv || status[0] != 0 || status[1] != 0 || status[2] != 0;
    rep->ok = bad ? 0 : 1;
}

__global__ void __launch_bounds__(32) k_step_finish(int S, const double* __restrict__ nu, int have_nu,
                                                    const int* __restrict__ status, StepReport* rep, LoopCtl* ctl) {
    double lo = 1.0, hi = 1.0;
    if (have_nu) {
        int bad = 0;
        for (int s = threadIdx.x; s < S; s += 32) {
            const double v = nu[s];
            bad |= !isfinite(v);
            lo = s == (int)threadIdx.x ? v : fmin(lo, v);
            hi = s == (int)threadIdx.x ? v : fmax(hi, v);
        }
        if ((int)threadIdx.x >= S) lo = hi = nu[0];
        bad = __any_sync(0xffffffffu, bad);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (bad) lo = hi = NAN;   // reported as a non-finite nu
    }
    if (threadIdx.x == 0) {
        rep->nu_min = lo;
        rep->nu_max = hi;
        for (int k = 0; k < 4; ++k) rep->status[k] = status[k];
        if (rep->ok) ctl->step++;
    }
}

static bool graph_usable(const gdc_ctx* c) {
    return c->p.graph && !c->prof_on && !c->fcm && (c->p.scheme == GDC_SCHEME_EM || c->p.divmode == GDC_DIV_RFD);
}

static void drop_graph(gdc_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_valid = 0;
}

static void graph_slip(gdc_ctx* c, const double* W, double* vb, int fixed, int run) {
    if (c->p.kT == 0.0) {
        cudaMemsetAsync(vb, 0, sizeof(double) * 3 * c->NBL, c->stream);
        return;
    }
    lanczos_sqrt_graph(c, W, vb, std::sqrt(2.0 * c->p.kT / c->p.dt), fixed, run);
}

// the launches of one step, in the order of one_step, for capture
static void enqueue_step_graph(gdc_ctx* c) {
    const double dt = c->p.dt;
    const unsigned long long* sd = &c->ctl->step;
    ++c->n_launch, k_step_begin<<<1, 32, 0, c->stream>>>(c->rep);
    launch_normals(c, 0, 0, c->W, sd);
    launch_normals(c, 0, 1, c->Wt, sd);
    const bool gdc_scheme = c->p.scheme != GDC_SCHEME_EM;
    if (!gdc_scheme) {
        load_at(c, c->Y, c->q);
        forces_at_loaded(c, c->FT);
        graph_slip(c, c->W, c->vb_m, 0, 2);
        launch_rhs(c, c->vb_m, c->FT, c->gm_b);
        gmres_solve_graph(c, c->gm_b, c->gm_x);
        launch_scatter_solution(c, c->gm_x, c->Vm, nullptr);
        ++c->n_launch, k_step_ok<<<1, 1, 0, c->stream>>>(c->rep, c->dev_status);
        launch_advance(c, c->Y, c->q, c->Vm, dt, nullptr, c->Y, c->q, &c->rep->ok);
    } else {
        load_at(c, c->Y, c->q);
        graph_slip(c, c->W, c->vb_n, 0, 0);
        launch_lsq(c, c->vb_n, c->calV);
        launch_perturb(c, c->Y, c->q, c->Wt, c->p.rfd_delta, c->Yt, c->qt);
        load_config(c, c->Yt, c->qt);
        cudaMemcpyAsync(c->lz_fix, c->lz_k, sizeof(int) * c->S, cudaMemcpyDeviceToDevice, c->stream);
        graph_slip(c, c->W, c->vb_t, 1, 1);
        launch_lsq(c, c->vb_t, c->calVt);
        launch_rfd_div(c, c->Wt, c->calV, c->calVt, c->p.rfd_delta, dt, c->nu);
        launch_advance(c, c->Y, c->q, c->calV, 0.5 * dt, nullptr, c->Ym, c->qm);
        load_at(c, c->Ym, c->qm);
        forces_at_loaded(c, c->FT);
        graph_slip(c, c->W, c->vb_m, 0, 2);
        launch_rhs(c, c->vb_m, c->FT, c->gm_b);
        gmres_solve_graph(c, c->gm_b, c->gm_x);
        launch_scatter_solution(c, c->gm_x, c->Vm, nullptr);
        ++c->n_launch, k_step_ok<<<1, 1, 0, c->stream>>>(c->rep, c->dev_status);
        launch_advance(c, c->Y, c->q, c->Vm, dt, c->nu, c->Y, c->q, &c->rep->ok);
    }
    if (c->have_trace) {
        const gdc_trace& t = c->trace;
        auto cp = [&](double* dst, const double* src, long long n) {
            if (dst) cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream);
        };
        cp(t.calV, c->calV, 6LL * c->NB);
        cp(t.nu, c->nu, c->S);
        cp(t.Ym, c->Ym, 3LL * c->NB);
        cp(t.qm, c->qm, 4LL * c->NB);
        cp(t.Vm, c->Vm, 6LL * c->NB);
        cp(t.vb_n, c->vb_n, 3LL * c->NBL);
        cp(t.vb_m, c->vb_m, 3LL * c->NBL);
        cp(t.FTm, c->FT, 6LL * c->NB);
    }
    ++c->n_launch, k_step_finish<<<1, 32, 0, c->stream>>>(c->S, c->nu, gdc_scheme ? 1 : 0, c->dev_status, c->rep,
                                                          c->ctl);
}

static gdc_status build_graph(gdc_ctx* c) {
    drop_graph(c);
    gdc_status st;
    for (cudaStream_t& s : c->cap_stream)
        if (!s && (st = cuda_check(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "capture stream")) != GDC_OK)
            return st;
    c->graph_loops.clear();
    c->cap_err = cudaSuccess;
    c->cap_depth = 0;
    const unsigned long long n0 = c->n_launch;
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream[0];
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) {
        enqueue_step_graph(c);
        e = cudaStreamEndCapture(c->stream, &g);
    }
    c->stream = user;
    c->graph_base_launches = c->n_launch - n0;
    c->n_launch = n0;
    if (e == cudaSuccess && c->cap_err != cudaSuccess) e = c->cap_err;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_check(c, e, "step graph capture");
    }
    c->graph = g;
    if ((st = cuda_check(c, cudaGraphInstantiate(&c->graph_exec, g, 0), "step graph instantiate")) != GDC_OK) {
        drop_graph(c);
        return st;
    }
    c->graph_valid = 1;
    return GDC_OK;
}

static gdc_status graph_step(gdc_ctx* c, gdc_step_info* info) {
    gdc_status st;
    if (!c->graph_valid && (st = build_graph(c)) != GDC_OK) return st;
    if (c->d_step_mirror != c->step) {
        const unsigned long long v = c->step;
        cudaError_t e = cudaMemcpyAsync(&c->ctl->step, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if ((st = cuda_check(c, e, "step counter upload")) != GDC_OK) return st;
        c->d_step_mirror = c->step;
    }
    StepReport r{};
    cudaError_t e = cudaGraphLaunch(c->graph_exec, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, c->rep, sizeof(r), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if ((st = cuda_check(c, e, "step graph")) != GDC_OK) return st;
    // kernels executed: those outside the loops plus each loop body times its iterations
    unsigned long long launches = c->graph_base_launches;
    for (const auto& lp : c->graph_loops) {
        const int slot = lp.first;
        const long long runs = slot < 3 ? r.lz_exec[slot]
                               : slot == REP_GM_TOTAL ? r.gm_total
                               : slot == REP_GM_OUTER ? r.gm_outer
                               : slot == REP_GM_DF    ? r.gm_df
                                                      : r.gm_outer - r.gm_df;
        launches += lp.second * (unsigned long long)std::max(0LL, runs);
    }
    c->n_launch += launches;
    if (r.ok) c->d_step_mirror = c->step + 1;
    gdc_step_info inf{};
    inf.step = c->step;
    for (int k = 0; k < 3; ++k) inf.lanczos_iters[k] = r.lz_iters[k];
    inf.lanczos_err = std::max(r.lz_err[0], r.lz_err[2]);
    inf.solve.iterations = r.gm_total;
    inf.solve.cycles = r.gm_cycles;
    inf.solve.residual = r.gm_residual;
    inf.solve.converged = r.gm_converged;
    if (c->p.precision == GDC_FP32_MIXED) {
        inf.solve.matvecs_fp32 = r.gm_total + (r.gm_outer - r.gm_df);
        inf.solve.matvecs_fp64 = r.gm_df;
    } else {
        inf.solve.matvecs_fp64 = r.gm_total + r.gm_outer;
    }
    inf.nu_min = r.nu_min;
    inf.nu_max = r.nu_max;
    const int matvecs = inf.lanczos_iters[0] + inf.lanczos_iters[1] + inf.lanczos_iters[2] + inf.solve.matvecs_fp32 +
                        inf.solve.matvecs_fp64;
    inf.pair_evals = (double)matvecs * c->pair_evals_per_matvec;
    // the host-driven path's checks, in its order
    if ((r.status[0] != 0 || r.status[1] != 0 || r.status[2] != 0) && clear_status(c) != GDC_OK) return GDC_ERR_CUDA;
    if (r.status[1] != 0) return fail(c, GDC_ERR_TIMEOUT, "a pair-kernel tile copy did not complete in time");
    if (r.status[2] != 0) return fail(c, GDC_ERR_NONFINITE, "a blob centre reached the wall (height <= a)");
    if (r.lz_notconv[0] || r.lz_notconv[2]) return fail(c, GDC_ERR_NOT_CONVERGED, "Lanczos reached lanczos_max_iter");
    if (r.gm_bad) return fail(c, GDC_ERR_NONFINITE, "mobility solve: non-finite residual");
    if (r.gm_notconv) return fail(c, GDC_ERR_NOT_CONVERGED, "mobility solve: GMRES reached gmres_max_iter");
    if (r.status[0] == 1) return fail(c, GDC_ERR_NONFINITE, "template RPY block is not positive definite");
    if (r.status[0] == 2) return fail(c, GDC_ERR_NOT_CONVERGED, "tridiagonal eigensolver did not converge");
    if (r.status[1] != 0) return fail(c, GDC_ERR_TIMEOUT, "a pair-kernel tile copy did not complete in time");
    if (!std::isfinite(inf.nu_min) || !std::isfinite(inf.nu_max)) return fail(c, GDC_ERR_NONFINITE, "non-finite nu");
    c->step++;
    if (info) *info = inf;
    return GDC_OK;
}

}  // namespace gdc

using namespace gdc;

extern "C" {

void gdc_debug_wait_polls(int polls) { g_wait_polls.store(polls); }

size_t gdc_workspace_bytes(const gdc_params* params, int n_templates, const int* tmpl_nblobs, int n_susp,
                           const long long* susp_body_off, const int* body_tmpl) {
    gdc_ctx tmp;
    if (build_host_layout(&tmp, params, n_templates, tmpl_nblobs, n_susp, susp_body_off, body_tmpl)) return 0;
    return carve(&tmp, nullptr);
}

gdc_status gdc_init(gdc_ctx** out, const gdc_params* params, int n_templates, const int* tmpl_nblobs,
                    const double* tmpl_xyz, int n_susp, const long long* susp_body_off, const int* body_tmpl,
                    double* Y, double* q, void* workspace, size_t workspace_bytes, void* stream) {
    if (!out) return GDC_ERR_INVALID_ARG;
    *out = nullptr;
    gdc_ctx* c = new (std::nothrow) gdc_ctx();
    if (!c) return GDC_ERR_INVALID_ARG;
    *out = c;
    c->stream = (cudaStream_t)stream;
    if (const char* m = build_host_layout(c, params, n_templates, tmpl_nblobs, n_susp, susp_body_off, body_tmpl))
        return fail(c, GDC_ERR_INVALID_ARG, m);
    if (!tmpl_xyz || !Y || !q || !workspace) return fail(c, GDC_ERR_INVALID_ARG, "NULL pointer argument");
    const size_t need = carve(c, nullptr);
    if (workspace_bytes < need)
        return fail(c, GDC_ERR_WORKSPACE, "workspace too small: need " + std::to_string(need) + " bytes");
    if (((uintptr_t)workspace) & 255) return fail(c, GDC_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    carve(c, workspace);
    c->Y = Y;
    c->q = q;
    // centre the templates on their blob centroids (Y_p is the centroid), body lengths L_p
    const long long nt = c->h_tmpl_off[c->T];
    c->h_tmpl_xyz.assign(tmpl_xyz, tmpl_xyz + 3 * nt);
    c->h_tmpl_L.assign(c->T, 0.0);
    for (int t = 0; t < c->T; ++t) {
        const int n = c->h_tmpl_n[t];
        double* b = c->h_tmpl_xyz.data() + 3LL * c->h_tmpl_off[t];
        double cen[3] = {0, 0, 0};
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k) {
                if (!std::isfinite(b[3 * i + k])) return fail(c, GDC_ERR_INVALID_ARG, "non-finite template coordinate");
                cen[k] += b[3 * i + k] / n;
            }
        double L = 0.0;
        for (int i = 0; i < n; ++i) {
            for (int k = 0; k < 3; ++k) b[3 * i + k] -= cen[k];
        }
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                double d2 = 0.0;
                for (int k = 0; k < 3; ++k) d2 += (b[3 * i + k] - b[3 * j + k]) * (b[3 * i + k] - b[3 * j + k]);
                L = std::max(L, std::sqrt(d2));
            }
        // L_p scales the translational RFD displacement (footnote to step 3); a single blob uses a
        c->h_tmpl_L[t] = L > 0.0 ? L : c->p.a;
    }
    gdc_status st;
    if ((st = upload_layout(c, c->h_tmpl_xyz.data())) != GDC_OK) return st;
    // state check on the host
    std::vector<double> hY(3LL * c->NB), hq(4LL * c->NB);
    cudaError_t e = cudaMemcpyAsync(hY.data(), Y, sizeof(double) * hY.size(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hq.data(), q, sizeof(double) * hq.size(), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if ((st = cuda_check(c, e, "state read")) != GDC_OK) return st;
    if ((st = check_state_host(c, hY.data(), hq.data())) != GDC_OK) return st;
    krylov_init_attributes();
    if (c->p.mobility == GDC_MOB_FCM) {
        // the FCM grid first: the preconditioner's template blocks are FCM blocks
        const gdc_fcm_params fp = fcm_params_of(c->p, c->NBL);
        if ((st = gdc_fcm_init(&c->fcm, &fp, c->fcm_ws, c->fcm_ws_bytes, c->stream)) != GDC_OK)
            return fail(c, st, "FCM context setup failed");
        if ((st = fcm_template_blocks(c)) != GDC_OK) return st;
    }
    launch_template_setup(c, c->fcm ? c->fcm_Mt : nullptr);
    if ((st = cuda_check(c, cudaGetLastError(), "template setup")) != GDC_OK) return st;
    if ((st = read_status(c)) != GDC_OK) return st;
    if ((st = sym_init_attributes(c)) != GDC_OK) return st;
    if ((st = dfsym_init_attributes(c)) != GDC_OK) return st;
    if (c->p.wall) {   // every blob must start above z = a
        load_at(c, c->Y, c->q);
        if ((st = read_status(c)) != GDC_OK) return st;
    }
    if (c->p.autotune && c->p.mobility == GDC_MOB_RPY) {   // the RPY pair kernels only
        load_at(c, c->Y, c->q);
        if ((st = autotune_pair_kernel(c)) != GDC_OK) return st;
    } else if ((st = default_pair_kernel(c)) != GDC_OK) {
        return st;
    }
    return GDC_OK;
}

void gdc_destroy(gdc_ctx* c) {
    if (!c) return;
    drop_graph(c);
    gdc_fcm_destroy(c->fcm);
    for (cudaStream_t s : c->cap_stream)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    delete c;
}

gdc_status gdc_profile(gdc_ctx* c, int enable) {
    if (!c) return GDC_ERR_INVALID_ARG;
    gdc_status st = cuda_check(c, cudaStreamSynchronize(c->stream), "profile");
    if (st != GDC_OK) return st;
    prof_flush(c);
    if (enable && c->prof_ev.empty()) {
        c->prof_ev.resize(2 * 1024);
        c->prof_kind.resize(1024);
        for (auto& e : c->prof_ev)
            if ((st = cuda_check(c, cudaEventCreate(&e), "event create")) != GDC_OK) return st;
    }
    c->prof_on = enable ? 1 : 0;
    c->n_launch = 0;
    for (int k = 0; k < 4; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_count[k] = 0;
    }
    return GDC_OK;
}

gdc_status gdc_profile_read(gdc_ctx* c, gdc_profile_info* out) {
    if (!c || !out) return c ? fail(c, GDC_ERR_INVALID_ARG, "NULL output") : GDC_ERR_INVALID_ARG;
    gdc_status st = cuda_check(c, cudaStreamSynchronize(c->stream), "profile read");
    if (st != GDC_OK) return st;
    prof_flush(c);
    out->launches = c->n_launch;
    out->rpy32_launches = c->prof_count[0];
    out->rpy64_launches = c->prof_count[1];
    out->force_launches = c->prof_count[2];
    out->rpy32_ms = c->prof_ms[0];
    out->rpy64_ms = c->prof_ms[1];
    out->force_ms = c->prof_ms[2];
    out->rpydf_launches = c->prof_count[3];
    out->rpydf_ms = c->prof_ms[3];
    out->pairs_per_product = c->pair_evals_per_matvec;
    out->targets_per_thread = c->mv_tpt;
    out->work_waves = c->mv_waves;
    out->autotune_ms = c->autotune_ms;
    out->pair_kernel = c->use_sym ? 2 : 1;
    out->sym_width = c->sym_width;
    out->min_blocks_per_sm = c->use_sym ? c->sym_minb : c->mv_minb;
    out->df_kernel = c->dfs_minb;
    double up = 0.0;
    for (int s = 0; s < c->S; ++s) {
        const double n = (double)(c->h_blob_off[s + 1] - c->h_blob_off[s]);
        up += n * (n + 1.0) / 2.0;
    }
    out->unique_pairs_per_product = up;
    return GDC_OK;
}

const char* gdc_last_error(const gdc_ctx* c) { return c ? c->err.c_str() : noalloc_last_error(); }

gdc_status gdc_set_params(gdc_ctx* c, const gdc_params* p) {
    if (!c) return GDC_ERR_INVALID_ARG;
    if (const char* m = validate_params(p)) return fail(c, GDC_ERR_INVALID_ARG, m);
    if (p->gmres_restart != c->p.gmres_restart || p->lanczos_max_iter != c->p.lanczos_max_iter)
        return fail(c, GDC_ERR_INVALID_ARG, "gmres_restart and lanczos_max_iter are fixed at init");
    if (p->a != c->p.a || p->eta != c->p.eta)
        return fail(c, GDC_ERR_INVALID_ARG, "a and eta are fixed at init (they shape the preconditioner)");
    if (p->mobility != c->p.mobility || p->box_L != c->p.box_L || p->fcm_N != c->p.fcm_N ||
        p->fcm_sigma != c->p.fcm_sigma || p->fcm_R_t != c->p.fcm_R_t)
        return fail(c, GDC_ERR_INVALID_ARG, "the mobility and its FCM grid are fixed at init");
    const unsigned long long seed = c->p.seed;
    const int pair_kernel = c->p.pair_kernel, df_kernel = c->p.df_kernel;
    c->p = *p;
    c->p.seed = seed;
    c->p.pair_kernel = pair_kernel;   // the pair kernels are chosen at init
    c->p.df_kernel = df_kernel;
    drop_graph(c);   // parameters are baked into the captured launches
    c->fcm_field_step = ~0ULL;   // an FCM field drawn with the old kT and dt is not reused
    return GDC_OK;
}

gdc_status gdc_mobility_solve(gdc_ctx* c, const double* FT, const double* vbrev, double* V, double* lambda,
                              gdc_solve_info* info) {
    if (!c) return GDC_ERR_INVALID_ARG;
    if (!FT || !V) return fail(c, GDC_ERR_INVALID_ARG, "FT and V are required");
    load_at(c, c->Y, c->q);
    launch_rhs(c, vbrev, FT, c->gm_b);
    gdc_solve_info inf{};
    gdc_status st = gmres_solve(c, c->gm_b, c->gm_x, &inf);
    launch_scatter_solution(c, c->gm_x, V, lambda);
    if (info) *info = inf;
    const gdc_status e2 = cuda_check(c, cudaStreamSynchronize(c->stream), "mobility solve");
    return e2 != GDC_OK ? e2 : settle(c, st);
}

gdc_status gdc_step(gdc_ctx* c, int nsteps, gdc_step_info* info) {
    if (!c) return GDC_ERR_INVALID_ARG;
    if (nsteps < 0) return fail(c, GDC_ERR_INVALID_ARG, "nsteps must be >= 0");
    for (int k = 0; k < nsteps; ++k) {
        const bool graph = graph_usable(c);
        gdc_status st = graph ? graph_step(c, info ? info + k : nullptr) : one_step(c, info ? info + k : nullptr);
        if (st != GDC_OK) return graph ? st : settle(c, st);
    }
    return GDC_OK;
}

gdc_status gdc_set_trace(gdc_ctx* c, const gdc_trace* t) {
    if (!c) return GDC_ERR_INVALID_ARG;
    if (t) {
        c->trace = *t;
        c->have_trace = 1;
    } else {
        c->have_trace = 0;
    }
    drop_graph(c);   // the trace copies are part of the captured step
    return GDC_OK;
}

gdc_status gdc_get_state(gdc_ctx* c, double* Y, double* q, unsigned long long* step) {
    if (!c) return GDC_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    if (Y) e = cudaMemcpyAsync(Y, c->Y, sizeof(double) * 3 * c->NB, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && q) e = cudaMemcpyAsync(q, c->q, sizeof(double) * 4 * c->NB, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (step) *step = c->step;
    return cuda_check(c, e, "get_state");
}

gdc_status gdc_set_state(gdc_ctx* c, const double* Y, const double* q, unsigned long long step) {
    if (!c) return GDC_ERR_INVALID_ARG;
    if (!Y || !q) return fail(c, GDC_ERR_INVALID_ARG, "Y and q are required");
    gdc_status st = check_state_host(c, Y, q);
    if (st != GDC_OK) return st;
    cudaError_t e = cudaMemcpyAsync(c->Y, Y, sizeof(double) * 3 * c->NB, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->q, q, sizeof(double) * 4 * c->NB, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->step = step;
    return cuda_check(c, e, "set_state");
}

gdc_status gdc_blob_positions(gdc_ctx* c, double* r) {
    if (!c || !r) return c ? fail(c, GDC_ERR_INVALID_ARG, "NULL output") : GDC_ERR_INVALID_ARG;
    load_at(c, c->Y, c->q);
    cudaMemcpyAsync(r, c->r, sizeof(double) * 3 * c->NBL, cudaMemcpyDeviceToDevice, c->stream);
    return cuda_check(c, cudaStreamSynchronize(c->stream), "blob positions");
}

gdc_status gdc_rpy_apply(gdc_ctx* c, int precision, const double* lam, double* u) {
    if (!c || !lam || !u) return c ? fail(c, GDC_ERR_INVALID_ARG, "NULL pointer") : GDC_ERR_INVALID_ARG;
    if (precision != GDC_FP64 && precision != GDC_FP32_MIXED && precision != GDC_DF64_RESIDUAL)
        return fail(c, GDC_ERR_INVALID_ARG, "unknown precision");
    load_at(c, c->Y, c->q);
    rpy_op(c, precision, lam, u);
    gdc_status st = cuda_check(c, cudaStreamSynchronize(c->stream), "rpy apply");
    return st != GDC_OK ? st : read_status(c);
}

gdc_status gdc_saddle_apply(gdc_ctx* c, int precision, const double* x, double* y) {
    if (!c || !x || !y) return c ? fail(c, GDC_ERR_INVALID_ARG, "NULL pointer") : GDC_ERR_INVALID_ARG;
    if (precision != GDC_FP64 && precision != GDC_FP32_MIXED && precision != GDC_DF64_RESIDUAL)
        return fail(c, GDC_ERR_INVALID_ARG, "unknown precision");
    load_at(c, c->Y, c->q);
    saddle_op(c, precision, x, y);
    gdc_status st = cuda_check(c, cudaStreamSynchronize(c->stream), "saddle apply");
    return st != GDC_OK ? st : read_status(c);
}

gdc_status gdc_precond_apply(gdc_ctx* c, const double* r, double* z) {
    if (!c || !r || !z) return c ? fail(c, GDC_ERR_INVALID_ARG, "NULL pointer") : GDC_ERR_INVALID_ARG;
    load_at(c, c->Y, c->q);
    launch_precond(c, r, z);
    return cuda_check(c, cudaStreamSynchronize(c->stream), "precond apply");
}

gdc_status gdc_brownian_slip(gdc_ctx* c, const double* W, double* vbrev, int* iters, double* err) {
    if (!c || !W || !vbrev) return c ? fail(c, GDC_ERR_INVALID_ARG, "NULL pointer") : GDC_ERR_INVALID_ARG;
    load_at(c, c->Y, c->q);
    gdc_status st = slip_at_loaded(c, W, vbrev, 0, iters, err);
    const gdc_status e2 = cuda_check(c, cudaStreamSynchronize(c->stream), "brownian slip");
    return e2 != GDC_OK ? e2 : settle(c, st);
}

gdc_status gdc_lsq_velocity(gdc_ctx* c, const double* vbrev, double* calV) {
    if (!c || !vbrev || !calV) return c ? fail(c, GDC_ERR_INVALID_ARG, "NULL pointer") : GDC_ERR_INVALID_ARG;
    load_at(c, c->Y, c->q);
    launch_lsq(c, vbrev, calV);
    return cuda_check(c, cudaStreamSynchronize(c->stream), "lsq velocity");
}

gdc_status gdc_forces(gdc_ctx* c, double* FT) {
    if (!c || !FT) return c ? fail(c, GDC_ERR_INVALID_ARG, "NULL pointer") : GDC_ERR_INVALID_ARG;
    load_at(c, c->Y, c->q);
    forces_at_loaded(c, FT);
    return cuda_check(c, cudaStreamSynchronize(c->stream), "forces");
}

gdc_status gdc_draw_normals(gdc_ctx* c, unsigned long long step, int stream, double* out) {
    if (!c || !out) return c ? fail(c, GDC_ERR_INVALID_ARG, "NULL pointer") : GDC_ERR_INVALID_ARG;
    if (stream != 0 && stream != 1) return fail(c, GDC_ERR_INVALID_ARG, "stream must be 0 (W) or 1 (W-tilde)");
    launch_normals(c, step, stream, out);
    return cuda_check(c, cudaStreamSynchronize(c->stream), "normals");
}

gdc_status gdc_saddle_offsets(const gdc_ctx* c, long long* off) {
    if (!c || !off) return GDC_ERR_INVALID_ARG;
    for (int s = 0; s <= c->S; ++s) off[s] = c->h_gm_off[s];
    return GDC_OK;
}

}  // extern "C"
