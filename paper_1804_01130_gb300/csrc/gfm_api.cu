// C ABI of libgfm (include/gfm.h): handle lifetime, argument checks, device
// workspace, launches of the assembly and solver kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "gfm_internal.h"
#include "gfm_setup.h"

struct gfm_ctx {
    int device = 0;
    int sm_count = 0;
    int smem_per_sm = 0, smem_optin = 0;
    int n = 0, F = 0;
    gfm::HostTables ht;
    // caller-order mesh copies
    int32_t *owner = nullptr, *neighbour = nullptr;
    double *Sf = nullptr, *C = nullptr;
    // renumbering + SELL
    int32_t *perm = nullptr, *iperm = nullptr;
    int32_t *slice_ptr = nullptr, *col = nullptr, *face = nullptr;
    double *val64 = nullptr;
    float *val32 = nullptr;
    // face arrays (caller order)
    double *lambda = nullptr, *gamma = nullptr, *jump = nullptr, *sigma = nullptr, *phi = nullptr;
    double *dl_dlam = nullptr;
    int8_t *kind = nullptr;
    // cell arrays
    double *alpha = nullptr;  // caller order copy (for the adjoint)
    double *b = nullptr, *diag = nullptr, *dinv = nullptr, *x64 = nullptr, *r64 = nullptr;
    double *p64 = nullptr, *q64 = nullptr, *rhs = nullptr, *tmp_user = nullptr, *tmp_user2 = nullptr;
    float2 *UP0 = nullptr, *UP1 = nullptr;
    float4 *Q0 = nullptr, *Q1 = nullptr;  // fused form: (q, t, p, region) per cell
    float *P32 = nullptr;
    float *R32 = nullptr, *S32 = nullptr, *E = nullptr, *dinv32 = nullptr;
    // two-level preconditioner (coarse space of connected one-phase regions)
    int32_t *cc_parent = nullptr, *cc_size = nullptr, *cc_cand = nullptr, *cc_counters = nullptr;
    int32_t *cc_bcount = nullptr, *cc_boff = nullptr;
    double *cc_epart = nullptr;
    int8_t *comp = nullptr;
    gfm::CrossFace *cross = nullptr;
    gfm::Coarse *coarse = nullptr;
    int max_cross = 0;
    int coarse_max = gfm::kMaxCoarse, coarse_min_size = 64;
    // batch of tanks (gfm_create_batched)
    bool batched = false;
    int T = 0, cta_grid = 0;
    gfm::BatchTables bt;
    int32_t *ftank = nullptr, *stank = nullptr, *tncell = nullptr;
    gfm::TankPhys *tphys = nullptr, *tphys_h = nullptr;
    gfm::DevParams *tprm = nullptr, *tprm_h = nullptr;
    int4 *cta = nullptr;
    int2 *tank_cta = nullptr;
    int32_t *tcoff = nullptr, *tioff = nullptr;  // [T+1] caller / internal cell offsets of the tanks
    gfm::TankCoarse *tco = nullptr;              // [T] coarse space of each tank
    std::vector<double> bweight;  // per-tank work weights of the CTA table (empty: by slices)
    gfm_solve_info *binfos = nullptr, *binfos_h = nullptr;
    // host-buffer entry point staging
    double *stage_alpha = nullptr, *stage_phi = nullptr, *stage_p = nullptr;
    // real pressure-equation inputs: face Rhie-Chow coefficient, explicit
    // non-orthogonal correction (allocated on first use)
    double *rau = nullptr;
    bool rau_set = false;
    double *nonorth_corr = nullptr, *phi_eff = nullptr, *grad_scr = nullptr;
    bool nonorth_active = false;
    // compact operator table for the streamed mixed pass (see Sell::ent):
    // usable when every neighbour offset fits 16 bits and the faces fall
    // into at most (kMaxDict - 1) / 2 classes of bit-identical c_f
    bool ct_ok = false, ent_valid = false;
    bool ct_pref = false;       // gfm_set_table: use the compact table when usable (off by default)
    bool force_stream = false;  // gfm_set_table: stream the tables even when they fit
    int n_cls = 0;
    uint32_t *ent = nullptr;
    int32_t *fcls = nullptr, *ctank = nullptr;
    double *ccls = nullptr;
    float *dict = nullptr;
    // control
    gfm::DevParams *prm = nullptr;
    unsigned *bar = nullptr;
    int *err = nullptr;
    double *partials = nullptr;
    gfm_solve_info *dinfo = nullptr;
    gfm_solve_info *hinfo = nullptr;  // pinned host
    int max_grid = 0;
    // state
    bool assembled = false;
    gfm_phys phys{};
    int ref_internal = -1;
    gfm_tuning tuning{512, 1, 1};
    bool profiling = false;
    gfm_profile prof{};
    cudaEvent_t ev[6] = {};
    bool ev_recorded[6] = {};
    std::string last_error;
};

namespace {

gfm_status fail(gfm_ctx *h, gfm_status s, const std::string &msg)
{
    if (h) h->last_error = msg;
    return s;
}

gfm_status cuda_fail(gfm_ctx *h, cudaError_t e, const char *where)
{
    return fail(h, GFM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GFM_CUDA(h, call)                                    \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

void free_all(gfm_ctx *h)
{
    void *ptrs[] = {h->owner, h->neighbour, h->Sf, h->C, h->perm, h->iperm, h->slice_ptr, h->col, h->face,
                    h->val64, h->val32, h->lambda, h->gamma, h->jump, h->sigma, h->phi, h->dl_dlam, h->kind,
                    h->alpha, h->b, h->diag, h->dinv, h->x64, h->r64, h->p64, h->q64, h->rhs, h->tmp_user,
                    h->tmp_user2, h->UP0, h->UP1, h->Q0, h->Q1, h->P32, h->R32, h->S32, h->E, h->dinv32, h->stage_alpha,
                    h->stage_phi, h->stage_p, h->prm, h->bar,
                    h->err, h->partials, h->dinfo, h->cc_parent, h->cc_size, h->cc_cand, h->cc_counters,
                    h->cc_bcount, h->cc_boff, h->cc_epart,
                    h->comp, h->cross, h->coarse, h->ftank, h->stank, h->tncell, h->tphys, h->tprm, h->cta,
                    h->tank_cta, h->binfos, h->tcoff, h->tioff, h->tco, h->rau, h->nonorth_corr, h->phi_eff,
                    h->grad_scr, h->ent, h->fcls, h->ctank, h->ccls, h->dict};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    void *hptrs[] = {h->hinfo, h->tphys_h, h->tprm_h, h->binfos_h};
    for (void *p : hptrs)
        if (p) cudaFreeHost(p);
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
}

gfm::Sell sell_of(gfm_ctx *h)
{
    gfm::Sell m;
    m.n = h->n;
    m.n_pad = h->ht.n_pad;
    m.n_slices = h->ht.n_slices;
    m.n_slots = h->ht.n_slots;
    m.slice_ptr = h->slice_ptr;
    m.col = h->col;
    m.face = h->face;
    m.val64 = h->val64;
    m.val32 = h->val32;
    m.ent = h->ent_valid ? h->ent : nullptr;
    m.dict = h->dict;
    m.n_dict = 2 * h->n_cls + 1;
    return m;
}

gfm_status check_opts(gfm_ctx *h, const gfm_solve_opts *o)
{
    if (!o) return fail(h, GFM_ERR_ARG, "opts is NULL");
    if (o->mode != GFM_FP64 && o->mode != GFM_MIXED) return fail(h, GFM_ERR_ARG, "unknown mode");
    if (!(o->rtol > 0.0) || !(o->rtol < 1.0)) return fail(h, GFM_ERR_ARG, "rtol must be in (0, 1)");
    if (o->mode == GFM_MIXED && (!(o->inner_rtol > 0.0) || !(o->inner_rtol < 1.0)))
        return fail(h, GFM_ERR_ARG, "inner_rtol must be in (0, 1)");
    if (o->max_iters < 0 || o->max_refine < 0) return fail(h, GFM_ERR_ARG, "negative iteration caps");
    if (!(o->timeout_ms > 0.0)) return fail(h, GFM_ERR_ARG, "timeout_ms must be > 0");
    return GFM_OK;
}

// Launch shape of a persistent solve and its shared-memory staging of the
// slice tables: each CTA keeps its slices' (base, width) and as many of its
// slots (neighbour + coefficient) as fit next to the other CTAs of its SM.
struct LaunchPlan {
    int grid = 0, threads = 0, cache_cap = 0, meta_slots = 0;
    int n_stages = 0, stage_slices = 0, stage_cap = 0;  // streamed tables (MIXED), 0 = not streamed
    bool ct = false;                                  // the stages hold the compact table
    bool fused = false;                               // MIXED: the one-pass, one-all-reduce form
    size_t dyn = 0;
};

gfm_status plan_launch(gfm_ctx *h, gfm::Mode mode, LaunchPlan *lp)
{
    const int t = h->tuning.threads;
    int per = h->tuning.ctas_per_sm;
    // the fused form (single meshes, MIXED) never uses the compact table
    const bool fused = !h->batched && mode == gfm::Mode::MIXED && h->tuning.form == 2;
    const void *k = h->batched ? gfm::batched_kernel(h->ht.max_width)
                               : gfm::solver_kernel(mode, h->ht.max_width, t, false, false, fused);
    cudaFuncAttributes fa;
    GFM_CUDA(h, cudaFuncGetAttributes(&fa, k));
    int occ0 = 0;
    GFM_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, k, t, 0));
    if (occ0 < 1) return fail(h, GFM_ERR_ARG, "solver kernel cannot run with this many threads per CTA");
    if (per > occ0) per = occ0;
    int grid = h->sm_count * per;
    if (grid > h->max_grid) grid = h->max_grid;
    // per-CTA budget: the SM's shared memory split between its CTAs
    long long budget = (long long)h->smem_per_sm / per - (long long)fa.sharedSizeBytes - 1024;
    budget = std::min<long long>(budget, (long long)h->smem_optin - (long long)fa.sharedSizeBytes);
    if (budget < 0) budget = 0;
    const int ns = h->ht.n_slices;
    int max_nsl = 0, max_slots = 0;
    if (h->batched) {
        if (h->cta_grid != grid) return fail(h, GFM_ERR_STATE, "batched CTA table out of date");
        std::vector<int32_t> cta4, tank2;
        std::string err;
        if (!gfm::plan_batch_ctas(h->bt, grid, cta4, tank2, err, h->bweight)) return fail(h, GFM_ERR_ARG, err);
        for (int b = 0; b < grid; ++b) {
            const int s0 = cta4[(size_t)b * 4 + 1], s1 = cta4[(size_t)b * 4 + 2];
            max_nsl = std::max(max_nsl, s1 - s0);
            max_slots = std::max(max_slots, h->ht.slice_ptr[(size_t)s1] - h->ht.slice_ptr[(size_t)s0]);
        }
        // the device re-plans the table as tanks finish: room for the
        // metadata of any range it can hand out
        max_nsl = std::max(max_nsl, gfm::batch_replan_max_slices(h->bt, grid));
    } else {
        for (int b = 0; b < grid; ++b) {
            const int s0 = (int)(((long long)ns * b) / grid), s1 = (int)(((long long)ns * (b + 1)) / grid);
            max_nsl = std::max(max_nsl, s1 - s0);
            max_slots = std::max(max_slots, h->ht.slice_ptr[(size_t)s1] - h->ht.slice_ptr[(size_t)s0]);
        }
    }
    const int meta_slots = (max_nsl + 1) & ~1;
    const long long meta_bytes = (long long)meta_slots * 8;
    const long long slot_bytes = 4 + (mode == gfm::Mode::FP64 ? 8 : 4);
    long long cap = budget > meta_bytes ? (budget - meta_bytes) / slot_bytes : 0;
    cap = std::min<long long>(cap, max_slots);
    cap &= ~3LL;
    if (h->force_stream && mode == gfm::Mode::MIXED && max_slots > 0) cap = 0;
    if (meta_bytes > budget) return fail(h, GFM_ERR_ARG, "mesh too large for this launch shape");
    // Tables that do not fit: the mixed operator pass streams them through a
    // ring of 3 (else 2) stages, each a whole number of pass rounds (a round
    // = the slices the CTA's warps take at once: 4 per warp for rows of <= 6
    // faces, else 2).
    int n_stages = 0, stage_slices = 0, stage_cap = 0;
    // the compact table streams 4 bytes per slot instead of 8, and stages
    // its dictionary after the ring
    const bool ct = mode == gfm::Mode::MIXED && h->ent_valid && h->ct_pref && !fused;
    const long long sbytes = ct ? 4 : 8;
    const long long dict_bytes = ct ? ((long long)(2 * h->n_cls + 1) * 4 + 15) / 16 * 16 : 0;
    if (mode == gfm::Mode::MIXED && cap < max_slots) {
        const int maxw = std::max(1, h->ht.max_width);
        const int unit = (maxw <= 6 ? 4 : 2) * (t / 32);
        const long long per_unit = (long long)unit * 32 * maxw * sbytes;
        const long long need = (max_nsl + unit - 1) / unit;
        for (int S = 3; S >= 2 && n_stages == 0; --S) {
            const long long m = std::min<long long>((budget - meta_bytes - dict_bytes) / (S * per_unit), need);
            if (m >= 1) {
                n_stages = S;
                stage_slices = (int)(unit * m);
                stage_cap = stage_slices * 32 * maxw;
            }
        }
        if (n_stages) cap = 0;
    }
    const size_t dyn = (size_t)(meta_bytes +
                                (n_stages ? (long long)n_stages * stage_cap * sbytes + dict_bytes : cap * slot_bytes));
    if (n_stages)
        k = h->batched ? gfm::batched_kernel(h->ht.max_width, true, ct)
                       : gfm::solver_kernel(mode, h->ht.max_width, t, true, ct, fused);
    GFM_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int occ = 0;
    GFM_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, t, dyn));
    if (occ < per) return fail(h, GFM_ERR_ARG, "launch shape cannot be co-resident with its shared-memory staging");
    lp->grid = grid;
    lp->threads = t;
    lp->cache_cap = (int)cap;
    lp->meta_slots = meta_slots;
    lp->n_stages = n_stages;
    lp->stage_slices = stage_slices;
    lp->stage_cap = stage_cap;
    lp->ct = ct && n_stages > 0;
    lp->fused = fused;
    lp->dyn = dyn;
    return GFM_OK;
}

void prof_record(gfm_ctx *h, int k, cudaStream_t s)
{
    if (h->profiling && cudaEventRecord(h->ev[k], s) == cudaSuccess) h->ev_recorded[k] = true;
}

// Elapsed time between two recorded events, 0 otherwise; never leaves a
// sticky runtime error behind.
float prof_elapsed(gfm_ctx *h, int a, int b)
{
    float ms = 0.0f;
    if (!h->ev_recorded[a] || !h->ev_recorded[b]) return 0.0f;
    if (cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0.0f;
    }
    return ms;
}

// Entry of every call that launches work: drop a stale error left by code
// outside the library so that it is not reported as this call's failure.
void clear_stale_error() { (void)cudaGetLastError(); }

// Enqueue one persistent solve of A x = rhs (internal order) writing the
// solution in caller order to out_user.  info_dev receives the result.
gfm_status enqueue_solve(gfm_ctx *h, const gfm_solve_opts *o, const double *rhs, double *out_user, int use_x0,
                         gfm_solve_info *info_dev, cudaStream_t s)
{
    const gfm::Mode mode = (o->mode == GFM_MIXED) ? gfm::Mode::MIXED : gfm::Mode::FP64;
    LaunchPlan lp;
    gfm_status st = plan_launch(h, mode, &lp);
    if (st != GFM_OK) return st;
    const int grid = lp.grid, threads = lp.threads;
    GFM_CUDA(h, cudaMemsetAsync(h->bar, 0, sizeof(unsigned), s));
    GFM_CUDA(h, cudaMemsetAsync(h->err, 0, sizeof(int), s));
    GFM_CUDA(h, cudaMemsetAsync(info_dev, 0, sizeof(gfm_solve_info), s));
    gfm::SolveArgs a{};
    a.m = sell_of(h);
    a.prm = h->prm;
    a.b = rhs;
    a.diag64 = h->diag;
    a.dinv64 = h->dinv;
    a.x64 = h->x64;
    a.r64 = h->r64;
    a.p64 = h->p64;
    a.q64 = h->q64;
    a.UP0 = h->UP0;
    a.UP1 = h->UP1;
    a.Q0 = h->Q0;
    a.Q1 = h->Q1;
    a.P32 = h->P32;
    a.R32 = h->R32;
    a.S32 = h->S32;
    a.E = h->E;
    a.dinv32 = h->dinv32;
    a.iperm = h->iperm;
    a.p_user = out_user;
    a.rtol = o->rtol;
    a.inner_rtol = o->inner_rtol;
    a.max_iters = o->max_iters;
    a.max_refine = o->max_refine;
    a.use_x0 = use_x0;
    a.budget_ns = (unsigned long long)(o->timeout_ms * 1e6);
    a.coarse = h->coarse;
    a.comp = h->comp;
    a.cross = h->cross;
    a.cache_cap = lp.cache_cap;
    a.meta_slots = lp.meta_slots;
    a.n_stages = lp.n_stages;
    a.stage_slices = lp.stage_slices;
    a.stage_cap = lp.stage_cap;
    a.bar = h->bar;
    a.err = h->err;
    a.partials = h->partials;
    a.info = info_dev;
    gfm::BatchArgs ba{};
    const void *kernel = gfm::solver_kernel(mode, h->ht.max_width, threads, lp.n_stages > 0, lp.ct, lp.fused);
    if (h->batched) {
        a.n_per_tank = h->tncell;
        a.prm = h->tprm;
        ba.T = h->T;
        ba.cta = h->cta;
        ba.tank_cta = h->tank_cta;
        ba.tprm = h->tprm;
        ba.infos = info_dev;
        ba.tco = h->tco;
        kernel = gfm::batched_kernel(h->ht.max_width, lp.n_stages > 0, lp.ct);
        GFM_CUDA(h, cudaMemsetAsync(info_dev, 0, sizeof(gfm_solve_info) * h->T, s));
    }
    void *args[] = {&a, &ba};
    prof_record(h, 2, s);
    GFM_CUDA(h, cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(threads), args, lp.dyn, s));
    prof_record(h, 3, s);
    h->prof.grid = grid;
    h->prof.threads = threads;
    h->prof.launches += 1;
    h->prof.launches_total += 1;
    return GFM_OK;
}

gfm_status finish_info(gfm_ctx *h, const gfm_solve_opts *o, gfm_solve_info *info, cudaStream_t s)
{
    if (o->info_on_device) return GFM_OK;
    if (h->batched) {
        GFM_CUDA(h, cudaMemcpyAsync(h->binfos_h, h->binfos, sizeof(gfm_solve_info) * h->T, cudaMemcpyDeviceToHost, s));
        GFM_CUDA(h, cudaStreamSynchronize(s));
        if (info) std::memcpy(info, h->binfos_h, sizeof(gfm_solve_info) * h->T);
        if (h->profiling) {
            h->prof.ms_solve = prof_elapsed(h, 2, 3);
            h->prof.ms_total = prof_elapsed(h, 4, 5);
        }
        gfm_status worst = GFM_OK;
        for (int t = 0; t < h->T; ++t)
            if (h->binfos_h[t].status != GFM_OK) {
                worst = (gfm_status)h->binfos_h[t].status;
                char buf[160];
                snprintf(buf, sizeof buf, "tank %d ended with %s after %d iterations", t, gfm_status_string(worst),
                         h->binfos_h[t].iters);
                h->last_error = buf;
            }
        return worst;
    }
    GFM_CUDA(h, cudaMemcpyAsync(h->hinfo, h->dinfo, sizeof(gfm_solve_info), cudaMemcpyDeviceToHost, s));
    GFM_CUDA(h, cudaStreamSynchronize(s));
    if (info) *info = *h->hinfo;
    if (h->profiling) {
        h->prof.ms_solve = prof_elapsed(h, 2, 3);
        h->prof.ms_total = prof_elapsed(h, 4, 5);
    }
    const gfm_status st = (gfm_status)h->hinfo->status;
    if (st != GFM_OK) {
        char buf[200];
        snprintf(buf, sizeof buf, "solve ended with %s after %d iterations (rel. residual %.3e)",
                 gfm_status_string(st), h->hinfo->iters, h->hinfo->rel_res_l2);
        h->last_error = buf;
    }
    return st;
}

gfm_status check_compat(gfm_ctx *h, cudaStream_t s)
{
    // Unpinned: the singular system needs sum(b) ~ 0.
    if (h->ref_internal >= 0) return GFM_OK;
    gfm::DevParams p;
    GFM_CUDA(h, cudaMemcpyAsync(&p, h->prm, sizeof p, cudaMemcpyDeviceToHost, s));
    GFM_CUDA(h, cudaStreamSynchronize(s));
    if (fabs(p.bsum) > 1e-12 * p.babs)
        return fail(h, GFM_ERR_INCOMPATIBLE, "unpinned system with incompatible source (sum(b) != 0)");
    return GFM_OK;
}

gfm_status init_device(gfm_ctx *h)
{
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess)
        return fail(h, GFM_ERR_CUDA, "no CUDA device");
    return GFM_OK;
}

// Device workspace and the mesh tables (h->n, h->F, h->ht set).
gfm_status alloc_upload(gfm_ctx *h, cudaStream_t s)
{
    const int n = h->n, F = h->F;
    const size_t np = (size_t)h->ht.n_pad, ns = (size_t)h->ht.n_slots;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gfm::solver_kernel(gfm::Mode::MIXED, h->ht.max_width, 32), 32, 0);
    h->max_grid = h->sm_count * (occ > 0 ? occ : 1);
    cudaError_t e = cudaSuccess;
#define A(ptr, cnt) \
    if (e == cudaSuccess) e = dalloc(&h->ptr, (cnt))
    A(owner, F); A(neighbour, F); A(Sf, 3 * (size_t)F); A(C, 3 * (size_t)n);
    A(perm, n); A(iperm, np); A(slice_ptr, (size_t)h->ht.n_slices + 1); A(col, ns); A(face, ns);
    A(val64, ns); A(val32, ns);
    A(lambda, F); A(gamma, F); A(jump, F); A(sigma, F); A(phi, F); A(dl_dlam, F); A(kind, F);
    A(alpha, n); A(b, np); A(diag, np); A(dinv, np); A(x64, np); A(r64, np); A(p64, np); A(q64, np);
    A(rhs, np); A(tmp_user, n); A(tmp_user2, n); A(UP0, np); A(UP1, np); A(Q0, np); A(Q1, np); A(P32, np); A(R32, np); A(S32, np); A(E, np);
    A(dinv32, np);
    A(stage_alpha, n); A(stage_phi, F); A(stage_p, n);
    A(prm, 1); A(bar, 1); A(err, 1); A(partials, 2 * (size_t)h->max_grid * gfm::kMaxReduce); A(dinfo, 1);
    h->max_cross = (int)std::min<long long>((long long)F, std::max<long long>(65536, (long long)F / 8));
    A(cc_parent, n); A(cc_size, n); A(cc_cand, gfm::kMaxCandidates); A(cc_counters, 2);
    A(cc_bcount, (F + 255) / 256); A(cc_boff, (F + 255) / 256);
    A(cc_epart, (size_t)gfm::kCoarseEParts * gfm::kMaxCoarse * gfm::kMaxCoarse);
    A(comp, np); A(cross, h->max_cross); A(coarse, 1);
#undef A
    if (e != cudaSuccess)
        return fail(h, e == cudaErrorMemoryAllocation ? GFM_ERR_NOMEM : GFM_ERR_CUDA,
                    std::string("device allocation: ") + cudaGetErrorString(e));
    if (cudaMallocHost((void **)&h->hinfo, sizeof(gfm_solve_info)) != cudaSuccess)
        return fail(h, GFM_ERR_NOMEM, "pinned host allocation");
    for (auto &ev : h->ev) cudaEventCreate(&ev);
    e = cudaMemcpyAsync(h->perm, h->ht.perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->iperm, h->ht.iperm.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->slice_ptr, h->ht.slice_ptr.data(), sizeof(int32_t) * (h->ht.n_slices + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->col, h->ht.col.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->face, h->ht.face.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s);
    // zero every vector once so padding lanes hold finite values
    double *zero_d[] = {h->b, h->diag, h->dinv, h->x64, h->r64, h->p64, h->q64, h->rhs};
    for (double *zp : zero_d)
        if (e == cudaSuccess) e = cudaMemsetAsync(zp, 0, sizeof(double) * np, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->comp, 0xff, np, s);  // -1: no coarse region
    if (e == cudaSuccess) e = cudaMemsetAsync(h->coarse, 0, sizeof(gfm::Coarse), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->UP0, 0, sizeof(float2) * np, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->UP1, 0, sizeof(float2) * np, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Q0, 0, sizeof(float4) * np, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Q1, 0, sizeof(float4) * np, s);
    float *zero_f[] = {h->R32, h->S32, h->E, h->dinv32};
    for (float *zp : zero_f)
        if (e == cudaSuccess) e = cudaMemsetAsync(zp, 0, sizeof(float) * np, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "uploading tables");
    return GFM_OK;
}

// Compact operator table (after the mesh is on the device).  Usable when
// every slot's neighbour lies within a signed 16-bit offset of its own cell
// and the faces fall into few classes of bit-identical c_f = S.S/S.d (per
// tank in a batch): off the interface a face's FP32 coefficient is then one
// of two dictionary values of its class, and each slot fits one word.  Not
// usable: the full table streams, nothing else changes.
gfm_status setup_compact(gfm_ctx *h, cudaStream_t s)
{
    h->ct_ok = false;
    const gfm::HostTables &ht = h->ht;
    for (int sl = 0; sl < ht.n_slices; ++sl) {
        const int base = ht.slice_ptr[(size_t)sl], w = (ht.slice_ptr[(size_t)sl + 1] - base) / gfm::kSlice;
        for (int k = 0; k < w; ++k)
            for (int l = 0; l < gfm::kSlice; ++l) {
                const size_t slot = (size_t)base + (size_t)k * gfm::kSlice + l;
                if (ht.face[slot] == 0) continue;
                const long long off = (long long)ht.col[slot] - ((long long)sl * gfm::kSlice + l);
                if (off < -32768 || off > 32767) return GFM_OK;
            }
    }
    const int F = h->F;
    double *dc = nullptr;
    if (dalloc(&dc, (size_t)F) != cudaSuccess) return fail(h, GFM_ERR_NOMEM, "compact table set-up");
    std::vector<double> c((size_t)F);
    cudaError_t e = gfm::launch_face_c(h->n, F, h->owner, h->neighbour, h->Sf, h->C, dc, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.data(), dc, sizeof(double) * F, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dc);
    if (e != cudaSuccess) return cuda_fail(h, e, "compact table set-up");
    const int max_cls = (gfm::kMaxDict - 1) / 2;
    std::vector<int32_t> fcls((size_t)F), ctank;
    std::vector<double> ccls;
    std::unordered_map<unsigned long long, int32_t> seen;
    int tank = -1;
    for (int f = 0; f < F; ++f) {
        const int t = h->batched ? h->bt.face_tank[(size_t)f] : 0;
        if (t != tank) {  // faces are grouped by tank: classes never span tanks
            seen.clear();
            tank = t;
        }
        unsigned long long bits;
        std::memcpy(&bits, &c[(size_t)f], sizeof(bits));
        auto it = seen.find(bits);
        if (it == seen.end()) {
            if ((int)ccls.size() >= max_cls) return GFM_OK;
            it = seen.emplace(bits, (int32_t)ccls.size()).first;
            ccls.push_back(c[(size_t)f]);
            ctank.push_back(t);
        }
        fcls[(size_t)f] = it->second;
    }
    const int ncls = (int)ccls.size();
    e = dalloc(&h->ent, (size_t)ht.n_slots);
    if (e == cudaSuccess) e = dalloc(&h->fcls, (size_t)F);
    if (e == cudaSuccess) e = dalloc(&h->ccls, (size_t)ncls);
    if (e == cudaSuccess) e = dalloc(&h->ctank, (size_t)ncls);
    if (e == cudaSuccess) e = dalloc(&h->dict, (size_t)(2 * ncls + 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->fcls, fcls.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->ccls, ccls.data(), sizeof(double) * ncls, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->ctank, ctank.data(), sizeof(int32_t) * ncls, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return fail(h, e == cudaErrorMemoryAllocation ? GFM_ERR_NOMEM : GFM_ERR_CUDA, "compact table set-up");
    h->n_cls = ncls;
    h->ct_ok = true;
    return GFM_OK;
}

// Batch-only workspace: tank of every face and slice, per-tank physics,
// pins, cell counts and results, CTA table.
gfm_status alloc_batch(gfm_ctx *h, cudaStream_t s)
{
    const int T = h->T;
    cudaError_t e = dalloc(&h->ftank, (size_t)h->F);
    if (e == cudaSuccess) e = dalloc(&h->stank, (size_t)h->ht.n_slices);
    if (e == cudaSuccess) e = dalloc(&h->tphys, (size_t)T);
    if (e == cudaSuccess) e = dalloc(&h->tprm, (size_t)T);
    if (e == cudaSuccess) e = dalloc(&h->tncell, (size_t)T);
    if (e == cudaSuccess) e = dalloc(&h->cta, (size_t)h->max_grid);
    if (e == cudaSuccess) e = dalloc(&h->tank_cta, (size_t)T);
    if (e == cudaSuccess) e = dalloc(&h->binfos, (size_t)T);
    if (e == cudaSuccess) e = dalloc(&h->tcoff, (size_t)T + 1);
    if (e == cudaSuccess) e = dalloc(&h->tioff, (size_t)T + 1);
    if (e == cudaSuccess) e = dalloc(&h->tco, (size_t)T);
    if (e != cudaSuccess) return fail(h, GFM_ERR_NOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
    if (cudaMallocHost((void **)&h->tphys_h, sizeof(gfm::TankPhys) * T) != cudaSuccess ||
        cudaMallocHost((void **)&h->tprm_h, sizeof(gfm::DevParams) * T) != cudaSuccess ||
        cudaMallocHost((void **)&h->binfos_h, sizeof(gfm_solve_info) * T) != cudaSuccess)
        return fail(h, GFM_ERR_NOMEM, "pinned host allocation");
    e = cudaMemcpyAsync(h->ftank, h->bt.face_tank.data(), sizeof(int32_t) * h->F, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->stank, h->bt.slice_tank.data(), sizeof(int32_t) * h->ht.n_slices, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->tncell, h->bt.ncell.data(), sizeof(int32_t) * T, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->tcoff, h->bt.coff.data(), sizeof(int32_t) * (T + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->tioff, h->bt.ioff.data(), sizeof(int32_t) * (T + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "uploading batch tables");
    return GFM_OK;
}

// CTA table of the batched solve for the current launch shape (synchronous).
gfm_status plan_batch(gfm_ctx *h)
{
    if (!h->batched) return GFM_OK;
    const int grid = std::min(h->sm_count * h->tuning.ctas_per_sm, h->max_grid);
    std::vector<int32_t> cta4, tank2;
    std::string err;
    if (!gfm::plan_batch_ctas(h->bt, grid, cta4, tank2, err, h->bweight)) return fail(h, GFM_ERR_ARG, err);
    cudaError_t e = cudaMemcpy(h->cta, cta4.data(), sizeof(int32_t) * cta4.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->tank_cta, tank2.data(), sizeof(int32_t) * tank2.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "uploading the CTA table");
    h->cta_grid = grid;
    return GFM_OK;
}

}  // namespace

extern "C" {

const char *gfm_status_string(gfm_status s)
{
    switch (s) {
    case GFM_OK: return "GFM_OK";
    case GFM_ERR_ARG: return "GFM_ERR_ARG";
    case GFM_ERR_CUDA: return "GFM_ERR_CUDA";
    case GFM_ERR_NOMEM: return "GFM_ERR_NOMEM";
    case GFM_ERR_NOT_CONVERGED: return "GFM_ERR_NOT_CONVERGED";
    case GFM_ERR_BREAKDOWN: return "GFM_ERR_BREAKDOWN";
    case GFM_ERR_TIMEOUT: return "GFM_ERR_TIMEOUT";
    case GFM_ERR_INCOMPATIBLE: return "GFM_ERR_INCOMPATIBLE";
    case GFM_ERR_STATE: return "GFM_ERR_STATE";
    }
    return "GFM_ERR_UNKNOWN";
}

const char *gfm_last_error(gfm_handle h) { return h ? h->last_error.c_str() : "NULL handle"; }

gfm_status gfm_default_opts(gfm_solve_opts *o)
{
    if (!o) return GFM_ERR_ARG;
    o->mode = GFM_FP64;
    o->rtol = 1e-10;
    o->inner_rtol = 1e-4;
    o->max_iters = 1000000;
    o->max_refine = 30;
    o->use_x0 = 0;
    o->info_on_device = 0;
    o->timeout_ms = 2000.0;
    return GFM_OK;
}

gfm_status gfm_create(const gfm_mesh *mesh, int32_t renumber, gfm_stream stream, gfm_handle *out)
{
    if (!out) return GFM_ERR_ARG;
    *out = nullptr;
    if (!mesh || !mesh->owner || !mesh->neighbour || !mesh->Sf || !mesh->C) return GFM_ERR_ARG;
    if (mesh->n_cells <= 0 || mesh->n_faces <= 0) return GFM_ERR_ARG;
    if (renumber < 0 || renumber > 2) return GFM_ERR_ARG;
    gfm_ctx *h = new (std::nothrow) gfm_ctx();
    if (!h) return GFM_ERR_NOMEM;
    clear_stale_error();
    cudaStream_t s = (cudaStream_t)stream;
    const int n = mesh->n_cells, F = mesh->n_faces;
    h->n = n;
    h->F = F;
    gfm_status st = init_device(h);
    do {
        if (st != GFM_OK) break;
        std::vector<int32_t> ho((size_t)F), hn((size_t)F);
        std::vector<double> hC;
        if (cudaMemcpyAsync(ho.data(), mesh->owner, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(hn.data(), mesh->neighbour, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess) {
            st = fail(h, GFM_ERR_CUDA, "reading owner/neighbour (must be device pointers)");
            break;
        }
        if (renumber == 2) {
            hC.resize((size_t)3 * n);
            if (cudaMemcpyAsync(hC.data(), mesh->C, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess) {
                st = fail(h, GFM_ERR_CUDA, "reading cell centres");
                break;
            }
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            st = fail(h, GFM_ERR_CUDA, "synchronising stream");
            break;
        }
        std::string err;
        if (!gfm::build_host_tables(n, F, ho.data(), hn.data(), hC.empty() ? nullptr : hC.data(), renumber, h->ht,
                                    err)) {
            st = fail(h, GFM_ERR_ARG, err);
            break;
        }
        h->ht.iperm.resize((size_t)h->ht.n_pad, -1);  // padding cells
        st = alloc_upload(h, s);
        if (st != GFM_OK) break;
        cudaError_t e = cudaMemcpyAsync(h->owner, mesh->owner, sizeof(int32_t) * F, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->neighbour, mesh->neighbour, sizeof(int32_t) * F, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->Sf, mesh->Sf, sizeof(double) * 3 * F, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->C, mesh->C, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = cuda_fail(h, e, "copying the mesh");
            break;
        }
        st = setup_compact(h, s);
    } while (0);
    if (st != GFM_OK) {
        fprintf(stderr, "gfm_create: %s\n", h->last_error.c_str());
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return GFM_OK;
}

gfm_status gfm_create_batched(const gfm_mesh *meshes, int32_t n_tanks, int32_t renumber, gfm_stream stream,
                              gfm_handle *out)
{
    if (!out) return GFM_ERR_ARG;
    *out = nullptr;
    if (!meshes || n_tanks <= 0 || n_tanks > gfm::kMaxTanks || renumber < 0 || renumber > 2) return GFM_ERR_ARG;
    for (int t = 0; t < n_tanks; ++t) {
        const gfm_mesh &m = meshes[t];
        if (!m.owner || !m.neighbour || !m.Sf || !m.C || m.n_cells <= 0 || m.n_faces <= 0) return GFM_ERR_ARG;
    }
    gfm_ctx *h = new (std::nothrow) gfm_ctx();
    if (!h) return GFM_ERR_NOMEM;
    clear_stale_error();
    cudaStream_t s = (cudaStream_t)stream;
    gfm_status st = init_device(h);
    do {
        if (st != GFM_OK) break;
        std::vector<std::vector<int32_t>> ho((size_t)n_tanks), hn((size_t)n_tanks);
        std::vector<std::vector<double>> hC((size_t)n_tanks);
        long long ncell = 0, nface = 0;
        for (int t = 0; t < n_tanks; ++t) {
            const gfm_mesh &m = meshes[t];
            ho[(size_t)t].resize((size_t)m.n_faces);
            hn[(size_t)t].resize((size_t)m.n_faces);
            cudaError_t e = cudaMemcpyAsync(ho[(size_t)t].data(), m.owner, sizeof(int32_t) * m.n_faces,
                                            cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hn[(size_t)t].data(), m.neighbour, sizeof(int32_t) * m.n_faces,
                                    cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && renumber == 2) {
                hC[(size_t)t].resize((size_t)3 * m.n_cells);
                e = cudaMemcpyAsync(hC[(size_t)t].data(), m.C, sizeof(double) * 3 * m.n_cells, cudaMemcpyDeviceToHost,
                                    s);
            }
            if (e != cudaSuccess) {
                st = cuda_fail(h, e, "reading tank meshes (must be device pointers)");
                break;
            }
            ncell += m.n_cells;
            nface += m.n_faces;
        }
        if (st != GFM_OK) break;
        if (ncell > INT32_MAX || nface > INT32_MAX) {
            st = fail(h, GFM_ERR_ARG, "batch too large");
            break;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            st = fail(h, GFM_ERR_CUDA, "synchronising stream");
            break;
        }
        std::vector<gfm::TankMesh> tm((size_t)n_tanks);
        for (int t = 0; t < n_tanks; ++t)
            tm[(size_t)t] = gfm::TankMesh{meshes[t].n_cells, meshes[t].n_faces, ho[(size_t)t].data(),
                                          hn[(size_t)t].data(), hC[(size_t)t].empty() ? nullptr : hC[(size_t)t].data()};
        std::string err;
        if (!gfm::build_batch_tables(tm, renumber, h->ht, h->bt, err)) {
            st = fail(h, GFM_ERR_ARG, err);
            break;
        }
        h->n = (int)ncell;
        h->F = (int)nface;
        h->batched = true;
        h->T = n_tanks;
        h->coarse_max = gfm::kTankCoarse;  // per tank: the water body and the air above it
        st = alloc_upload(h, s);
        if (st != GFM_OK) break;
        st = alloc_batch(h, s);
        if (st != GFM_OK) break;
        // caller-order concatenated mesh: indices offset by the tanks' cell offsets
        std::vector<int32_t> co((size_t)h->F), cn((size_t)h->F);
        for (int t = 0; t < n_tanks; ++t) {
            const int32_t c0 = h->bt.coff[(size_t)t], f0 = h->bt.foff[(size_t)t];
            for (int f = 0; f < meshes[t].n_faces; ++f) {
                co[(size_t)f0 + f] = ho[(size_t)t][(size_t)f] + c0;
                cn[(size_t)f0 + f] = hn[(size_t)t][(size_t)f] + c0;
            }
        }
        cudaError_t e = cudaMemcpyAsync(h->owner, co.data(), sizeof(int32_t) * h->F, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->neighbour, cn.data(), sizeof(int32_t) * h->F, cudaMemcpyHostToDevice, s);
        for (int t = 0; t < n_tanks && e == cudaSuccess; ++t) {
            const int nt = meshes[t].n_cells, ft = meshes[t].n_faces;
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
                e = cudaMemcpyAsync(h->Sf + (size_t)k * h->F + h->bt.foff[(size_t)t], meshes[t].Sf + (size_t)k * ft,
                                    sizeof(double) * ft, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(h->C + (size_t)k * h->n + h->bt.coff[(size_t)t], meshes[t].C + (size_t)k * nt,
                                        sizeof(double) * nt, cudaMemcpyDeviceToDevice, s);
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = cuda_fail(h, e, "copying the tank meshes");
            break;
        }
        st = setup_compact(h, s);
        if (st != GFM_OK) break;
        st = plan_batch(h);
    } while (0);
    if (st != GFM_OK) {
        fprintf(stderr, "gfm_create_batched: %s\n", h->last_error.c_str());
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return GFM_OK;
}

gfm_status gfm_destroy(gfm_handle h)
{
    if (!h) return GFM_ERR_ARG;
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return GFM_OK;
}

gfm_status gfm_assemble(gfm_handle h, const double *alpha, const double *phi, const gfm_phys *phys,
                        gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    clear_stale_error();
    if (!alpha || !phi || !phys) return fail(h, GFM_ERR_ARG, "alpha, phi and phys must be non-NULL");
    const int nphys = h->batched ? h->T : 1;
    for (int t = 0; t < nphys; ++t) {
        const gfm_phys &ph = phys[t];
        const int ncell_t = h->batched ? h->bt.ncell[(size_t)t] : h->n;
        if (!(ph.rho_a > 0.0) || !(ph.rho_w >= ph.rho_a) || !std::isfinite(ph.rho_w))
            return fail(h, GFM_ERR_ARG, "densities must satisfy 0 < rho_a <= rho_w");
        if (ph.ref_cell < -1 || ph.ref_cell >= ncell_t) return fail(h, GFM_ERR_ARG, "ref_cell out of range");
        if (h->batched && ph.ref_cell < 0) return fail(h, GFM_ERR_ARG, "every tank of a batch needs a pinned cell");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(ph.g[k])) return fail(h, GFM_ERR_ARG, "g must be finite");
    }
    cudaStream_t s = (cudaStream_t)stream;
    h->prof.launches = 0;
    prof_record(h, 4, s);
    prof_record(h, 0, s);
    h->phys = *phys;
    h->ref_internal = (h->batched || phys->ref_cell >= 0) ? (h->batched ? 0 : h->ht.perm[(size_t)phys->ref_cell]) : -1;
    GFM_CUDA(h, cudaMemcpyAsync(h->alpha, alpha, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s));
    GFM_CUDA(h, cudaMemcpyAsync(h->phi, phi, sizeof(double) * h->F, cudaMemcpyDeviceToDevice, s));
    GFM_CUDA(h, cudaMemsetAsync(h->prm, 0, sizeof(gfm::DevParams), s));
    if (h->batched) {
        for (int t = 0; t < h->T; ++t) {
            const gfm_phys &ph = phys[t];
            gfm::TankPhys tp{ph.rho_w, ph.rho_a, ph.g[0], ph.g[1], ph.g[2], ph.ref_value,
                             h->ht.perm[(size_t)h->bt.coff[(size_t)t] + ph.ref_cell], 0};
            h->tphys_h[t] = tp;
            gfm::DevParams dp{};
            dp.ref = tp.ref;
            h->tprm_h[t] = dp;
        }
        GFM_CUDA(h, cudaMemcpyAsync(h->tphys, h->tphys_h, sizeof(gfm::TankPhys) * h->T, cudaMemcpyHostToDevice, s));
        GFM_CUDA(h, cudaMemcpyAsync(h->tprm, h->tprm_h, sizeof(gfm::DevParams) * h->T, cudaMemcpyHostToDevice, s));
    }
    gfm::FaceArgs fa;
    fa.n = h->n;
    fa.F = h->F;
    fa.owner = h->owner;
    fa.neighbour = h->neighbour;
    fa.Sf = h->Sf;
    fa.C = h->C;
    fa.alpha = h->alpha;
    fa.phi = h->phi;
    fa.rho_w = phys->rho_w;
    fa.rho_a = phys->rho_a;
    fa.g0 = phys->g[0];
    fa.g1 = phys->g[1];
    fa.g2 = phys->g[2];
    fa.lambda = h->lambda;
    fa.gamma = h->gamma;
    fa.jump = h->jump;
    fa.sigma = h->sigma;
    fa.kind = h->kind;
    fa.ftank = h->batched ? h->ftank : nullptr;
    fa.tphys = h->batched ? h->tphys : nullptr;
    fa.rau = h->rau_set ? h->rau : nullptr;
    GFM_CUDA(h, gfm::launch_faces(fa, s));
    h->nonorth_active = false;
    // the compact table's codes hold only while gamma_f off the interface is
    // c_f / rho of the phase, i.e. without a face Rhie-Chow coefficient
    const bool use_ct = h->ct_ok && !h->rau_set;
    int launched = 2;
    if (use_ct) {
        gfm::DictArgs da{};
        da.n_cls = h->n_cls;
        da.ccls = h->ccls;
        da.ctank = h->batched ? h->ctank : nullptr;
        da.tphys = h->batched ? h->tphys : nullptr;
        da.rho_w = phys->rho_w;
        da.rho_a = phys->rho_a;
        da.dict = h->dict;
        GFM_CUDA(h, gfm::launch_dict(da, s));
        ++launched;
    }
    gfm::CellArgs ca{};
    ca.m = sell_of(h);
    ca.gamma = h->gamma;
    ca.sigma = h->sigma;
    ca.ref = h->ref_internal;
    ca.ref_value = phys->ref_value;
    ca.b = h->b;
    ca.diag = h->diag;
    ca.dinv = h->dinv;
    ca.dinv32 = h->dinv32;
    ca.prm = h->prm;
    ca.iperm = h->iperm;
    ca.stank = h->batched ? h->stank : nullptr;
    ca.tphys = h->batched ? h->tphys : nullptr;
    ca.tprm = h->batched ? h->tprm : nullptr;
    ca.ent = use_ct ? h->ent : nullptr;
    ca.fcls = h->fcls;
    ca.kind = h->kind;
    ca.pad_code = 2 * h->n_cls;
    GFM_CUDA(h, gfm::launch_cells(ca, s));
    h->ent_valid = use_ct;
    {
        gfm::CoarseArgs co{};
        co.n = h->n;
        co.F = h->F;
        co.n_pad = h->ht.n_pad;
        co.owner = h->owner;
        co.neighbour = h->neighbour;
        co.perm = h->perm;
        co.kind = h->kind;
        co.gamma = h->gamma;
        co.ref = h->ref_internal;
        co.max_k = h->coarse_max;
        co.min_size = h->coarse_min_size;
        co.max_cross = h->max_cross;
        co.prm = h->prm;
        co.parent = h->cc_parent;
        co.csize = h->cc_size;
        co.cand = h->cc_cand;
        co.counters = h->cc_counters;
        co.bcount = h->cc_bcount;
        co.boff = h->cc_boff;
        co.epart = h->cc_epart;
        co.comp = h->comp;
        co.cross = h->cross;
        co.coarse = h->coarse;
        if (h->batched) {  // one coarse space per tank
            co.T = h->T;
            co.coff = h->tcoff;
            co.ioff = h->tioff;
            co.tprm = h->tprm;
            co.tco = h->tco;
            co.max_k = std::min(h->coarse_max, gfm::kTankCoarse);
        }
        GFM_CUDA(h, gfm::launch_coarse(co, s, &launched));
    }
    if (h->ref_internal < 0) {  // only an unpinned system needs sum(b) for its compatibility test
        GFM_CUDA(h, gfm::launch_bsums(h->b, h->n, h->prm, s));
        ++launched;
    }
    prof_record(h, 1, s);
    h->prof.launches += launched;
    h->prof.launches_total += launched;
    h->assembled = true;
    return GFM_OK;
}

gfm_status gfm_export_system(gfm_handle h, double *lambda, double *gamma, double *jump, double *diag, double *b,
                             gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    if (!h->assembled) return fail(h, GFM_ERR_STATE, "export before assemble");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t F = (size_t)h->F;
    if (lambda) GFM_CUDA(h, cudaMemcpyAsync(lambda, h->lambda, sizeof(double) * F, cudaMemcpyDeviceToDevice, s));
    if (gamma) GFM_CUDA(h, cudaMemcpyAsync(gamma, h->gamma, sizeof(double) * F, cudaMemcpyDeviceToDevice, s));
    if (jump) GFM_CUDA(h, cudaMemcpyAsync(jump, h->jump, sizeof(double) * F, cudaMemcpyDeviceToDevice, s));
    // internal -> caller order: out[iperm[i]] = v[i]; done with a host-side
    // copy of the permutation via two gathers is not needed: iperm's inverse
    // is perm, so out[c] = v[perm[c]] is a gather by perm.
    if (diag) GFM_CUDA(h, gfm::launch_gather(h->diag, h->perm, diag, h->n, h->n, s));
    if (b) GFM_CUDA(h, gfm::launch_gather(h->b, h->perm, b, h->n, h->n, s));
    return GFM_OK;
}

gfm_status gfm_solve(gfm_handle h, const gfm_solve_opts *opts, double *p, double *phi_corr, gfm_solve_info *info,
                     gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    gfm_status st = check_opts(h, opts);
    if (st != GFM_OK) return st;
    if (!p) return fail(h, GFM_ERR_ARG, "p must be non-NULL");
    if (opts->info_on_device && !info) return fail(h, GFM_ERR_ARG, "info_on_device needs a device info pointer");
    if (!h->assembled) return fail(h, GFM_ERR_STATE, "solve before assemble");
    clear_stale_error();
    cudaStream_t s = (cudaStream_t)stream;
    if (!opts->info_on_device) {
        st = check_compat(h, s);
        if (st != GFM_OK) return st;
    }
    h->prof.launches = 0;
    if (h->batched && opts->mode != GFM_MIXED)
        return fail(h, GFM_ERR_ARG, "a batched handle solves in GFM_MIXED mode");
    prof_record(h, 4, s);
    gfm_solve_info *idev = opts->info_on_device ? info : (h->batched ? h->binfos : h->dinfo);
    st = enqueue_solve(h, opts, h->b, p, opts->use_x0, idev, s);
    if (st != GFM_OK) return st;
    if (phi_corr) {
        GFM_CUDA(h, gfm::launch_corrected_flux(h->F, h->owner, h->neighbour, h->gamma, h->jump,
                                               h->nonorth_active ? h->phi_eff : h->phi, p, phi_corr, s));
        h->prof.launches += 1;
        h->prof.launches_total += 1;
    }
    prof_record(h, 5, s);
    if (opts->info_on_device) return GFM_OK;
    return finish_info(h, opts, info, s);
}

gfm_status gfm_solve_adjoint(gfm_handle h, const gfm_solve_opts *opts, const double *p, const double *dL_dp,
                             double *dL_dphi, double *dL_dalpha, double *mu, gfm_solve_info *info, gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    gfm_status st = check_opts(h, opts);
    if (st != GFM_OK) return st;
    if (!p || !dL_dp || !dL_dphi || !dL_dalpha) return fail(h, GFM_ERR_ARG, "p, dL_dp, dL_dphi, dL_dalpha required");
    if (opts->info_on_device && !info) return fail(h, GFM_ERR_ARG, "info_on_device needs a device info pointer");
    if (!h->assembled) return fail(h, GFM_ERR_STATE, "adjoint before assemble");
    if (h->batched) return fail(h, GFM_ERR_ARG, "the adjoint solve takes a single-mesh handle");
    clear_stale_error();
    cudaStream_t s = (cudaStream_t)stream;
    h->prof.launches = 0;
    prof_record(h, 4, s);
    GFM_CUDA(h, gfm::launch_gather(dL_dp, h->iperm, h->rhs, h->n, h->ht.n_pad, s));
    double *mu_out = mu ? mu : h->tmp_user;
    gfm_solve_info *idev = opts->info_on_device ? info : h->dinfo;
    st = enqueue_solve(h, opts, h->rhs, mu_out, 0, idev, s);
    if (st != GFM_OK) return st;
    gfm::AdjointArgs a;
    a.n = h->n;
    a.F = h->F;
    a.owner = h->owner;
    a.neighbour = h->neighbour;
    a.C = h->C;
    a.alpha = h->alpha;
    a.lambda = h->lambda;
    a.gamma = h->gamma;
    a.jump = h->jump;
    a.kind = h->kind;
    a.rho_w = h->phys.rho_w;
    a.rho_a = h->phys.rho_a;
    a.g0 = h->phys.g[0];
    a.g1 = h->phys.g[1];
    a.g2 = h->phys.g[2];
    a.p = p;
    a.mu = mu_out;
    a.dL_dphi = dL_dphi;
    a.dL_dlam = h->dl_dlam;
    a.m = sell_of(h);
    a.perm = h->perm;
    a.iperm = h->iperm;
    a.dL_dalpha = dL_dalpha;
    GFM_CUDA(h, gfm::launch_adjoint_faces(a, s));
    GFM_CUDA(h, gfm::launch_adjoint_cells(a, s));
    h->prof.launches += 3;
    h->prof.launches_total += 3;
    prof_record(h, 5, s);
    if (opts->info_on_device) return GFM_OK;
    return finish_info(h, opts, info, s);
}

gfm_status gfm_solve_host(gfm_handle h, const double *alpha_host, const double *phi_host, const gfm_phys *phys,
                          const gfm_solve_opts *opts, double *p_host, gfm_solve_info *info, gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    if (!alpha_host || !phi_host || !p_host) return fail(h, GFM_ERR_ARG, "host buffers must be non-NULL");
    gfm_status st = check_opts(h, opts);
    if (st != GFM_OK) return st;
    if (opts->info_on_device) return fail(h, GFM_ERR_ARG, "gfm_solve_host reports info on the host");
    if (h->batched) return fail(h, GFM_ERR_ARG, "gfm_solve_host takes a single-mesh handle");
    clear_stale_error();
    cudaStream_t s = (cudaStream_t)stream;
    GFM_CUDA(h, cudaMemcpyAsync(h->stage_alpha, alpha_host, sizeof(double) * h->n, cudaMemcpyHostToDevice, s));
    GFM_CUDA(h, cudaMemcpyAsync(h->stage_phi, phi_host, sizeof(double) * h->F, cudaMemcpyHostToDevice, s));
    if (opts->use_x0)
        GFM_CUDA(h, cudaMemcpyAsync(h->stage_p, p_host, sizeof(double) * h->n, cudaMemcpyHostToDevice, s));
    st = gfm_assemble(h, h->stage_alpha, h->stage_phi, phys, stream);
    if (st != GFM_OK) return st;
    st = check_compat(h, s);
    if (st != GFM_OK) return st;
    st = enqueue_solve(h, opts, h->b, h->stage_p, opts->use_x0, h->dinfo, s);
    if (st != GFM_OK) return st;
    GFM_CUDA(h, cudaMemcpyAsync(p_host, h->stage_p, sizeof(double) * h->n, cudaMemcpyDeviceToHost, s));
    prof_record(h, 5, s);
    return finish_info(h, opts, info, s);
}

gfm_status gfm_gradient(gfm_handle h, const double *p, const double *V, const double *xf, double *grad,
                        const double *phi, double *U, gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    if (!p || !V) return fail(h, GFM_ERR_ARG, "p and V must be non-NULL");
    if (!grad && !U) return fail(h, GFM_ERR_ARG, "nothing to compute: grad and U are both NULL");
    if (U && !phi) return fail(h, GFM_ERR_ARG, "U needs the face flux phi");
    if (grad && !h->assembled) return fail(h, GFM_ERR_STATE, "gradient before assemble");
    clear_stale_error();
    cudaStream_t s = (cudaStream_t)stream;
    gfm::GradArgs a{};
    a.m = sell_of(h);
    a.n = h->n;
    a.F = h->F;
    a.iperm = h->iperm;
    a.owner = h->owner;
    a.neighbour = h->neighbour;
    a.Sf = h->Sf;
    a.C = h->C;
    a.V = V;
    a.xf = xf;
    a.lambda = h->lambda;
    a.jump = h->jump;
    a.p = p;
    a.phi = phi;
    a.rho_w = h->phys.rho_w;
    a.rho_a = h->phys.rho_a;
    a.stank = h->batched ? h->stank : nullptr;
    a.tphys = h->batched ? h->tphys : nullptr;
    a.grad = grad;
    a.U = U;
    GFM_CUDA(h, gfm::launch_gradient(a, s));
    h->prof.launches = 1;
    h->prof.launches_total += 1;
    return GFM_OK;
}

gfm_status gfm_set_rau(gfm_handle h, const double *rau, gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    clear_stale_error();
    if (!rau) {
        h->rau_set = false;
        return GFM_OK;
    }
    if (!h->rau) {
        cudaError_t e = dalloc(&h->rau, (size_t)h->F);
        if (e != cudaSuccess) return fail(h, GFM_ERR_NOMEM, "allocating the face coefficient");
    }
    GFM_CUDA(h, cudaMemcpyAsync(h->rau, rau, sizeof(double) * h->F, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    h->rau_set = true;
    return GFM_OK;
}

gfm_status gfm_nonorth_correct(gfm_handle h, const double *p, const double *V, const double *xf, double *corr,
                               gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    if (!p || !V) return fail(h, GFM_ERR_ARG, "p and V must be non-NULL");
    if (!h->assembled) return fail(h, GFM_ERR_STATE, "non-orthogonal correction before assemble");
    clear_stale_error();
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->grad_scr) {
        cudaError_t e = dalloc(&h->grad_scr, 3 * (size_t)h->n);
        if (e == cudaSuccess) e = dalloc(&h->nonorth_corr, (size_t)h->F);
        if (e == cudaSuccess) e = dalloc(&h->phi_eff, (size_t)h->F);
        if (e != cudaSuccess) return fail(h, GFM_ERR_NOMEM, "allocating the correction workspace");
    }
    gfm::GradArgs ga{};
    ga.m = sell_of(h);
    ga.n = h->n;
    ga.F = h->F;
    ga.iperm = h->iperm;
    ga.owner = h->owner;
    ga.neighbour = h->neighbour;
    ga.Sf = h->Sf;
    ga.C = h->C;
    ga.V = V;
    ga.xf = xf;
    ga.lambda = h->lambda;
    ga.jump = h->jump;
    ga.p = p;
    ga.rho_w = h->phys.rho_w;
    ga.rho_a = h->phys.rho_a;
    ga.stank = h->batched ? h->stank : nullptr;
    ga.tphys = h->batched ? h->tphys : nullptr;
    ga.grad = h->grad_scr;
    GFM_CUDA(h, gfm::launch_gradient(ga, s));
    gfm::NonorthArgs na{};
    na.n = h->n;
    na.F = h->F;
    na.owner = h->owner;
    na.neighbour = h->neighbour;
    na.Sf = h->Sf;
    na.C = h->C;
    na.xf = xf;
    na.rau = h->rau_set ? h->rau : nullptr;
    na.G = h->grad_scr;
    na.phi = h->phi;
    na.gamma = h->gamma;
    na.jump = h->jump;
    na.corr = h->nonorth_corr;
    na.phi_eff = h->phi_eff;
    na.sigma = h->sigma;
    GFM_CUDA(h, gfm::launch_nonorth(na, s));
    // the cell sums again: b from the corrected sigma (diag and the tables
    // are rewritten with the same values; the compact table is unchanged)
    gfm::CellArgs ca{};
    ca.m = sell_of(h);
    ca.gamma = h->gamma;
    ca.sigma = h->sigma;
    ca.ref = h->ref_internal;
    ca.ref_value = h->phys.ref_value;
    ca.b = h->b;
    ca.diag = h->diag;
    ca.dinv = h->dinv;
    ca.dinv32 = h->dinv32;
    ca.prm = h->prm;
    ca.iperm = h->iperm;
    ca.stank = h->batched ? h->stank : nullptr;
    ca.tphys = h->batched ? h->tphys : nullptr;
    ca.tprm = h->batched ? h->tprm : nullptr;
    GFM_CUDA(h, gfm::launch_cells(ca, s));
    int launched = 3;
    if (h->ref_internal < 0) {
        GFM_CUDA(h, gfm::launch_bsums(h->b, h->n, h->prm, s));
        ++launched;
    }
    if (corr) GFM_CUDA(h, cudaMemcpyAsync(corr, h->nonorth_corr, sizeof(double) * h->F, cudaMemcpyDeviceToDevice, s));
    h->nonorth_active = true;
    h->prof.launches = launched;
    h->prof.launches_total += launched;
    return GFM_OK;
}

gfm_status gfm_piso_step(gfm_handle h, const gfm_solve_opts *opts, int32_t n_solves, int32_t n_nonorth,
                         const double *alpha, const double *phi_star, const gfm_phys *phys, double *p, double *phi_corr,
                         const double *V, const double *xf, double *grad, double *U, gfm_solve_info *info,
                         gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    if (!opts || !alpha || !phi_star || !phys || !p || !info) return fail(h, GFM_ERR_ARG, "NULL argument");
    if (!opts->info_on_device) return fail(h, GFM_ERR_ARG, "gfm_piso_step reports info on the device");
    if (n_solves < 1 || n_nonorth < 0) return fail(h, GFM_ERR_ARG, "n_solves >= 1, n_nonorth >= 0");
    if ((n_nonorth > 0 || grad || U) && !V) return fail(h, GFM_ERR_ARG, "the gradient steps need V");
    const bool batched = h->batched;
    cudaStream_t s = (cudaStream_t)stream;
    gfm_solve_opts o = *opts;
    for (int k = 0; k < n_solves; ++k) {
        // corrector k: the pressure equation of its predicted flux, solved
        // from the last corrector's p_d (the first from opts->use_x0).  alpha
        // is the step's, so after the first full assembly only the source
        // changes: sigma and the cell sums again, bit-identical to a full
        // assembly with this flux
        gfm_status st = GFM_OK;
        if (k == 0) {
            st = gfm_assemble(h, alpha, phi_star, phys, stream);
            if (st != GFM_OK) return st;
        } else {
            const double *phik = phi_star + (size_t)k * h->F;
            GFM_CUDA(h, cudaMemcpyAsync(h->phi, phik, sizeof(double) * h->F, cudaMemcpyDeviceToDevice, s));
            GFM_CUDA(h, gfm::launch_sigma(h->F, h->phi, h->gamma, h->jump, h->sigma, s));
            gfm::CellArgs ca{};
            ca.m = sell_of(h);
            ca.gamma = h->gamma;
            ca.sigma = h->sigma;
            ca.ref = h->ref_internal;
            ca.ref_value = h->phys.ref_value;
            ca.b = h->b;
            ca.diag = h->diag;
            ca.dinv = h->dinv;
            ca.dinv32 = h->dinv32;
            ca.prm = h->prm;
            ca.iperm = h->iperm;
            ca.stank = batched ? h->stank : nullptr;
            ca.tphys = batched ? h->tphys : nullptr;
            ca.tprm = batched ? h->tprm : nullptr;
            GFM_CUDA(h, gfm::launch_cells(ca, s));
            if (h->ref_internal < 0) GFM_CUDA(h, gfm::launch_bsums(h->b, h->n, h->prm, s));
            h->nonorth_active = false;
        }
        o.use_x0 = (k == 0) ? opts->use_x0 : 1;
        const bool last = k == n_solves - 1;
        gfm_solve_info *ik = info + (size_t)k * (batched ? h->T : 1);
        st = gfm_solve(h, &o, p, (last && n_nonorth == 0) ? phi_corr : nullptr, ik, stream);
        if (st != GFM_OK) return st;
        for (int j = 0; j < n_nonorth; ++j) {
            st = gfm_nonorth_correct(h, p, V, xf, nullptr, stream);
            if (st != GFM_OK) return st;
            o.use_x0 = 1;
            st = gfm_solve(h, &o, p, (last && j == n_nonorth - 1) ? phi_corr : nullptr, ik, stream);
            if (st != GFM_OK) return st;
        }
    }
    if (grad || U) {
        if (U && !phi_corr) return fail(h, GFM_ERR_ARG, "U needs phi_corr");
        return gfm_gradient(h, p, V, xf, grad, phi_corr, U, stream);
    }
    return GFM_OK;
}

gfm_status gfm_iso_advect(gfm_handle h, const double *alpha, const double *phi, double dt, const int32_t *fv_ptr,
                          const double *fv_xyz, int32_t nvt, const double *xf, const int8_t *has_iso,
                          const double *xS, const double *nS, const double *UnS, const double *V, double *integral,
                          double *dV, double *alpha_new, gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    if (!alpha || !phi || !fv_ptr || !fv_xyz || !xf || !has_iso || !xS || !nS || !UnS || !dV)
        return fail(h, GFM_ERR_ARG, "NULL argument");
    if (alpha_new && !V) return fail(h, GFM_ERR_ARG, "the alpha update needs V");
    if (!(dt >= 0.0) || !std::isfinite(dt) || nvt < 3) return fail(h, GFM_ERR_ARG, "dt >= 0 and nvt >= 3");
    clear_stale_error();
    gfm::IsoArgs a{};
    a.m = sell_of(h);
    a.n = h->n;
    a.F = h->F;
    a.nvt = nvt;
    a.iperm = h->iperm;
    a.owner = h->owner;
    a.neighbour = h->neighbour;
    a.alpha = alpha;
    a.phi = phi;
    a.dt = dt;
    a.fv_ptr = fv_ptr;
    a.fv_xyz = fv_xyz;
    a.xf = xf;
    a.has_iso = has_iso;
    a.xS = xS;
    a.nS = nS;
    a.UnS = UnS;
    a.V = V;
    a.integral = integral;
    a.dV = dV;
    a.alpha_new = alpha_new;
    GFM_CUDA(h, gfm::launch_iso(a, (cudaStream_t)stream));
    const int launched = alpha_new ? 2 : 1;
    h->prof.launches = launched;
    h->prof.launches_total += launched;
    return GFM_OK;
}

gfm_status gfm_set_table(gfm_handle h, int32_t compact, int32_t force_stream)
{
    if (!h) return GFM_ERR_ARG;
    h->ct_pref = compact != 0;
    h->force_stream = force_stream != 0;
    return GFM_OK;
}

gfm_status gfm_get_table(gfm_handle h, int32_t *compact_usable, int32_t *n_classes, int32_t *compact_valid)
{
    if (!h) return GFM_ERR_ARG;
    if (compact_usable) *compact_usable = h->ct_ok ? 1 : 0;
    if (n_classes) *n_classes = h->n_cls;
    if (compact_valid) *compact_valid = h->ent_valid ? 1 : 0;
    return GFM_OK;
}

gfm_status gfm_set_tuning(gfm_handle h, const gfm_tuning *t)
{
    if (!h || !t) return GFM_ERR_ARG;
    gfm_tuning nt = h->tuning;
    if (t->threads) nt.threads = t->threads;
    if (t->ctas_per_sm) nt.ctas_per_sm = t->ctas_per_sm;
    if (t->form) nt.form = t->form;
    if (nt.threads < 32 || nt.threads > gfm::solver_max_threads() || nt.threads % 32 || nt.ctas_per_sm < 1)
        return fail(h, GFM_ERR_ARG, "threads must be a multiple of 32 in [32, 1024], ctas_per_sm >= 1");
    if (nt.form != 1 && nt.form != 2) return fail(h, GFM_ERR_ARG, "form must be 1 (two passes) or 2 (fused)");
    if (nt.form == 2 && h->batched) return fail(h, GFM_ERR_ARG, "the batched solve has the two-pass form only");
    if (h->sm_count * nt.ctas_per_sm > h->max_grid) return fail(h, GFM_ERR_ARG, "grid larger than workspace");
    const gfm_tuning old = h->tuning;
    h->tuning = nt;
    if (h->batched && plan_batch(h) != GFM_OK) {
        h->tuning = old;
        plan_batch(h);
        return fail(h, GFM_ERR_ARG, "launch shape has fewer CTAs than tanks");
    }
    for (gfm::Mode m : {gfm::Mode::FP64, gfm::Mode::MIXED}) {
        int occ = 0;
        const void *k = gfm::solver_kernel(m, h->ht.max_width, nt.threads, false, false, nt.form == 2);
        GFM_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, nt.threads, 0));
        LaunchPlan lp;
        if (occ < nt.ctas_per_sm || plan_launch(h, m, &lp) != GFM_OK) {
            h->tuning = old;
            plan_batch(h);
            return fail(h, GFM_ERR_ARG, "launch shape cannot be co-resident");
        }
    }
    return GFM_OK;
}

gfm_status gfm_autotune(gfm_handle h, const gfm_solve_opts *opts, int32_t trials, gfm_tuning *chosen, float *best_ms,
                        gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    gfm_status st = check_opts(h, opts);
    if (st != GFM_OK) return st;
    if (trials < 1 || trials > 64) return fail(h, GFM_ERR_ARG, "trials must be in [1, 64]");
    if (!h->assembled) return fail(h, GFM_ERR_STATE, "autotune before assemble");
    if (h->batched && opts->mode != GFM_MIXED) return fail(h, GFM_ERR_ARG, "a batched handle solves in GFM_MIXED mode");
    clear_stale_error();
    cudaStream_t s = (cudaStream_t)stream;
    gfm_solve_opts o = *opts;
    o.use_x0 = 0;
    o.info_on_device = 1;
    gfm_solve_info *idev = h->batched ? h->binfos : h->dinfo;
    const int nrec = h->batched ? h->T : 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GFM_CUDA(h, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(h, GFM_ERR_CUDA, "cudaEventCreate");
    }
    // median time of `trials` solves with the current shape and table; ms = 0
    // when a solve fails (the candidate is then dropped)
    auto time_it = [&](float &ms, std::vector<int32_t> *iters) -> gfm_status {
        std::vector<float> t;
        ms = 0.0f;
        for (int k = 0; k < trials; ++k) {
            GFM_CUDA(h, cudaEventRecord(e0, s));
            if (gfm_solve(h, &o, h->tmp_user, nullptr, idev, stream) != GFM_OK) return GFM_OK;
            GFM_CUDA(h, cudaEventRecord(e1, s));
            GFM_CUDA(h, cudaEventSynchronize(e1));
            float x = 0.0f;
            GFM_CUDA(h, cudaEventElapsedTime(&x, e0, e1));
            t.push_back(x);
        }
        std::vector<gfm_solve_info> rec((size_t)nrec);
        GFM_CUDA(h, cudaMemcpy(rec.data(), idev, sizeof(gfm_solve_info) * nrec, cudaMemcpyDeviceToHost));
        for (const auto &r : rec)
            if (r.status != GFM_OK) return GFM_OK;
        if (iters) {
            iters->clear();
            for (const auto &r : rec) iters->push_back(r.iters);
        }
        std::sort(t.begin(), t.end());
        ms = t[t.size() / 2];
        return GFM_OK;
    };
    const gfm_tuning start = h->tuning;
    const std::vector<double> start_w = h->bweight;
    // shapes within 512 threads' worth of registers per SM (the solvers use
    // 128 registers a thread)
    const int shapes[][2] = {{512, 1}, {256, 2}, {128, 4}, {384, 1}, {256, 1}};
    std::vector<gfm_tuning> cands;
    // a single mesh in MIXED mode also tries the fused form with every shape
    const int n_forms = (!h->batched && opts->mode == GFM_MIXED) ? 2 : 1;
    for (int f = 1; f <= n_forms; ++f)
        for (const auto &sh : shapes) cands.push_back(gfm_tuning{sh[0], sh[1], f});
    gfm_tuning best = start;
    std::vector<double> best_w = start_w;
    float best_t = 0.0f;
    std::vector<int32_t> best_iters;
    for (const gfm_tuning &c : cands) {
        if (gfm_set_tuning(h, &c) != GFM_OK) continue;
        float ms = 0.0f;
        std::vector<int32_t> it;
        st = time_it(ms, &it);
        if (st != GFM_OK) break;
        if (ms > 0.0f && (best_t == 0.0f || ms < best_t)) {
            best_t = ms;
            best = c;
            best_iters = it;
        }
    }
    if (st == GFM_OK && h->batched && best_t > 0.0f && gfm_set_tuning(h, &best) == GFM_OK) {
        // the tank table weighted by the iterations each tank took
        h->bweight.assign(best_iters.begin(), best_iters.end());
        float ms = 0.0f;
        if (plan_batch(h) == GFM_OK) st = time_it(ms, nullptr);
        if (st == GFM_OK && ms > 0.0f && ms < best_t) {
            best_t = ms;
            best_w = h->bweight;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GFM_OK) return st;
    h->bweight = best_t > 0.0f ? best_w : start_w;
    const gfm_tuning keep = best_t > 0.0f ? best : start;
    st = gfm_set_tuning(h, &keep);
    if (st != GFM_OK) return st;
    if (best_t == 0.0f) return fail(h, GFM_ERR_NOT_CONVERGED, "no launch shape solved the system");
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return GFM_OK;
}

gfm_status gfm_get_tuning(gfm_handle h, gfm_tuning *t)
{
    if (!h || !t) return GFM_ERR_ARG;
    *t = h->tuning;
    return GFM_OK;
}

gfm_status gfm_set_coarse(gfm_handle h, int32_t max_vectors, int32_t min_size)
{
    if (!h) return GFM_ERR_ARG;
    if (max_vectors < 0 || max_vectors > gfm::kMaxCoarse || min_size < 1)
        return fail(h, GFM_ERR_ARG, "max_vectors must be in [0, 8] and min_size >= 1");
    h->coarse_max = max_vectors;
    h->coarse_min_size = min_size;
    return GFM_OK;
}

gfm_status gfm_get_coarse(gfm_handle h, int32_t *n_vectors, int32_t *n_regions, int32_t *sizes, gfm_stream stream)
{
    if (!h) return GFM_ERR_ARG;
    gfm::Coarse co;
    cudaStream_t s = (cudaStream_t)stream;
    GFM_CUDA(h, cudaMemcpyAsync(&co, h->coarse, sizeof co, cudaMemcpyDeviceToHost, s));
    if (h->batched) {  // vectors summed over the tanks; sizes of the first tanks' vectors
        std::vector<gfm::TankCoarse> tc((size_t)h->T);
        GFM_CUDA(h, cudaMemcpyAsync(tc.data(), h->tco, sizeof(gfm::TankCoarse) * h->T, cudaMemcpyDeviceToHost, s));
        GFM_CUDA(h, cudaStreamSynchronize(s));
        int nv = 0;
        for (const auto &t : tc)
            for (int k = 0; k < t.K; ++k) {
                if (sizes && nv < gfm::kMaxCoarse) sizes[nv] = t.sizes[k];
                ++nv;
            }
        if (sizes)
            for (int k = nv; k < gfm::kMaxCoarse; ++k) sizes[k] = 0;
        if (n_vectors) *n_vectors = nv;
        if (n_regions) *n_regions = co.n_cand;
        return GFM_OK;
    }
    GFM_CUDA(h, cudaStreamSynchronize(s));
    if (n_vectors) *n_vectors = co.K;
    if (n_regions) *n_regions = co.n_cand;
    if (sizes)
        for (int k = 0; k < gfm::kMaxCoarse; ++k) sizes[k] = k < co.K ? co.sizes[k] : 0;
    return GFM_OK;
}

gfm_status gfm_set_profiling(gfm_handle h, int32_t on)
{
    if (!h) return GFM_ERR_ARG;
    h->profiling = on != 0;
    return GFM_OK;
}

gfm_status gfm_get_profile(gfm_handle h, gfm_profile *out)
{
    if (!h || !out) return GFM_ERR_ARG;
    if (h->profiling) {
        for (int k = 0; k < 6; ++k)
            if (h->ev_recorded[k]) cudaEventSynchronize(h->ev[k]);
        h->prof.ms_assemble = prof_elapsed(h, 0, 1);
        h->prof.ms_solve = prof_elapsed(h, 2, 3);
        h->prof.ms_total = prof_elapsed(h, 4, 5);
        (void)cudaGetLastError();
    }
    *out = h->prof;
    return GFM_OK;
}

gfm_status gfm_get_sizes(gfm_handle h, int32_t *n_cells, int32_t *n_faces, int32_t *n_tanks)
{
    if (!h) return GFM_ERR_ARG;
    if (n_cells) *n_cells = h->n;
    if (n_faces) *n_faces = h->F;
    if (n_tanks) *n_tanks = h->batched ? h->T : 1;
    return GFM_OK;
}

gfm_status gfm_get_permutation(gfm_handle h, int32_t *perm_host)
{
    if (!h || !perm_host) return GFM_ERR_ARG;
    std::memcpy(perm_host, h->ht.perm.data(), sizeof(int32_t) * (size_t)h->n);
    return GFM_OK;
}

}  // extern "C"
