// C ABI of libgfm (include/gfm.h): handle lifetime, argument checks, device
// workspace, launches of the assembly and solver kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gfm_internal.h"
#include "gfm_setup.h"

struct gfm_ctx {
    int device = 0;
    int sm_count = 0;
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
    float *R32 = nullptr, *S32 = nullptr, *E = nullptr, *dinv32 = nullptr;
    // host-buffer entry point staging
    double *stage_alpha = nullptr, *stage_phi = nullptr, *stage_p = nullptr;
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
    gfm_tuning tuning{512, 1};
    bool profiling = false;
    gfm_profile prof{};
    cudaEvent_t ev[6] = {};
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
                    h->tmp_user2, h->UP0, h->UP1, h->R32, h->S32, h->E, h->dinv32, h->stage_alpha, h->stage_phi, h->stage_p, h->prm, h->bar,
                    h->err, h->partials, h->dinfo};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->hinfo) cudaFreeHost(h->hinfo);
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

gfm_status grid_shape(gfm_ctx *h, gfm::Mode mode, int *grid, int *threads)
{
    int t = h->tuning.threads, per = h->tuning.ctas_per_sm;
    int occ = 0;
    GFM_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gfm::solver_kernel(mode, h->ht.max_width, t), t, 0));
    if (occ < 1) return fail(h, GFM_ERR_ARG, "solver kernel cannot run with this many threads per CTA");
    if (per > occ) per = occ;
    *grid = h->sm_count * per;
    if (*grid > h->max_grid) *grid = h->max_grid;
    *threads = t;
    return GFM_OK;
}

void prof_record(gfm_ctx *h, int k, cudaStream_t s)
{
    if (h->profiling) cudaEventRecord(h->ev[k], s);
}

// Enqueue one persistent solve of A x = rhs (internal order) writing the
// solution in caller order to out_user.  info_dev receives the result.
gfm_status enqueue_solve(gfm_ctx *h, const gfm_solve_opts *o, const double *rhs, double *out_user, int use_x0,
                         gfm_solve_info *info_dev, cudaStream_t s)
{
    const gfm::Mode mode = (o->mode == GFM_MIXED) ? gfm::Mode::MIXED : gfm::Mode::FP64;
    int grid = 0, threads = 0;
    gfm_status st = grid_shape(h, mode, &grid, &threads);
    if (st != GFM_OK) return st;
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
    a.bar = h->bar;
    a.err = h->err;
    a.partials = h->partials;
    a.info = info_dev;
    void *args[] = {&a};
    prof_record(h, 2, s);
    GFM_CUDA(h, cudaLaunchCooperativeKernel(gfm::solver_kernel(mode, h->ht.max_width, threads), dim3(grid), dim3(threads), args, 0, s));
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
    GFM_CUDA(h, cudaMemcpyAsync(h->hinfo, h->dinfo, sizeof(gfm_solve_info), cudaMemcpyDeviceToHost, s));
    GFM_CUDA(h, cudaStreamSynchronize(s));
    if (info) *info = *h->hinfo;
    if (h->profiling) {
        cudaEventElapsedTime(&h->prof.ms_solve, h->ev[2], h->ev[3]);
        cudaEventElapsedTime(&h->prof.ms_total, h->ev[4], h->ev[5]);
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
    cudaStream_t s = (cudaStream_t)stream;
    const int n = mesh->n_cells, F = mesh->n_faces;
    h->n = n;
    h->F = F;
    gfm_status st = GFM_OK;
    do {
        if (cudaGetDevice(&h->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
            st = GFM_ERR_CUDA;
            h->last_error = "no CUDA device";
            break;
        }
        std::vector<int32_t> ho((size_t)F), hn((size_t)F);
        std::vector<double> hC;
        if (cudaMemcpyAsync(ho.data(), mesh->owner, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(hn.data(), mesh->neighbour, sizeof(int32_t) * F, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess) {
            st = GFM_ERR_CUDA;
            h->last_error = "reading owner/neighbour (must be device pointers)";
            break;
        }
        if (renumber == 2) {
            hC.resize((size_t)3 * n);
            if (cudaMemcpyAsync(hC.data(), mesh->C, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess) {
                st = GFM_ERR_CUDA;
                h->last_error = "reading cell centres";
                break;
            }
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            st = GFM_ERR_CUDA;
            h->last_error = "synchronising stream";
            break;
        }
        std::string err;
        if (!gfm::build_host_tables(n, F, ho.data(), hn.data(), hC.empty() ? nullptr : hC.data(), renumber, h->ht,
                                    err)) {
            st = GFM_ERR_ARG;
            h->last_error = err;
            break;
        }
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
        A(rhs, np); A(tmp_user, n); A(tmp_user2, n); A(UP0, np); A(UP1, np); A(R32, np); A(S32, np); A(E, np);
        A(dinv32, np);
        A(stage_alpha, n); A(stage_phi, F); A(stage_p, n);
        A(prm, 1); A(bar, 1); A(err, 1); A(partials, 2 * (size_t)h->max_grid * 4); A(dinfo, 1);
#undef A
        if (e != cudaSuccess) {
            st = (e == cudaErrorMemoryAllocation) ? GFM_ERR_NOMEM : GFM_ERR_CUDA;
            h->last_error = std::string("device allocation: ") + cudaGetErrorString(e);
            break;
        }
        if (cudaMallocHost((void **)&h->hinfo, sizeof(gfm_solve_info)) != cudaSuccess) {
            st = GFM_ERR_NOMEM;
            h->last_error = "pinned host allocation";
            break;
        }
        for (auto &ev : h->ev) cudaEventCreate(&ev);
        // iperm padded with the padding cells' own index
        std::vector<int32_t> ip(h->ht.iperm);
        ip.resize(np);
        for (size_t i = (size_t)n; i < np; ++i) ip[i] = (int32_t)i;
        e = cudaMemcpyAsync(h->owner, mesh->owner, sizeof(int32_t) * F, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->neighbour, mesh->neighbour, sizeof(int32_t) * F, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->Sf, mesh->Sf, sizeof(double) * 3 * F, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->C, mesh->C, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->perm, h->ht.perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->iperm, ip.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->slice_ptr, h->ht.slice_ptr.data(), sizeof(int32_t) * (h->ht.n_slices + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->col, h->ht.col.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->face, h->ht.face.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s);
        // zero every vector once so padding lanes hold finite values
        double *zero_d[] = {h->b, h->diag, h->dinv, h->x64, h->r64, h->p64, h->q64, h->rhs};
        for (double *zp : zero_d)
            if (e == cudaSuccess) e = cudaMemsetAsync(zp, 0, sizeof(double) * np, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->UP0, 0, sizeof(float2) * np, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->UP1, 0, sizeof(float2) * np, s);
        float *zero_f[] = {h->R32, h->S32, h->E, h->dinv32};
        for (float *zp : zero_f)
            if (e == cudaSuccess) e = cudaMemsetAsync(zp, 0, sizeof(float) * np, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = GFM_ERR_CUDA;
            h->last_error = std::string("uploading tables: ") + cudaGetErrorString(e);
            break;
        }
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
    if (!alpha || !phi || !phys) return fail(h, GFM_ERR_ARG, "alpha, phi and phys must be non-NULL");
    if (!(phys->rho_a > 0.0) || !(phys->rho_w >= phys->rho_a) || !std::isfinite(phys->rho_w))
        return fail(h, GFM_ERR_ARG, "densities must satisfy 0 < rho_a <= rho_w");
    if (phys->ref_cell < -1 || phys->ref_cell >= h->n) return fail(h, GFM_ERR_ARG, "ref_cell out of range");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(phys->g[k])) return fail(h, GFM_ERR_ARG, "g must be finite");
    cudaStream_t s = (cudaStream_t)stream;
    h->prof.launches = 0;
    prof_record(h, 4, s);
    prof_record(h, 0, s);
    h->phys = *phys;
    h->ref_internal = phys->ref_cell >= 0 ? h->ht.perm[(size_t)phys->ref_cell] : -1;
    GFM_CUDA(h, cudaMemcpyAsync(h->alpha, alpha, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s));
    GFM_CUDA(h, cudaMemcpyAsync(h->phi, phi, sizeof(double) * h->F, cudaMemcpyDeviceToDevice, s));
    GFM_CUDA(h, cudaMemsetAsync(h->prm, 0, sizeof(gfm::DevParams), s));
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
    GFM_CUDA(h, gfm::launch_faces(fa, s));
    gfm::CellArgs ca;
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
    GFM_CUDA(h, gfm::launch_cells(ca, s));
    int launched = 2;
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
    cudaStream_t s = (cudaStream_t)stream;
    if (!opts->info_on_device) {
        st = check_compat(h, s);
        if (st != GFM_OK) return st;
    }
    h->prof.launches = 0;
    prof_record(h, 4, s);
    gfm_solve_info *idev = opts->info_on_device ? info : h->dinfo;
    st = enqueue_solve(h, opts, h->b, p, opts->use_x0, idev, s);
    if (st != GFM_OK) return st;
    if (phi_corr) {
        GFM_CUDA(h, gfm::launch_corrected_flux(h->F, h->owner, h->neighbour, h->gamma, h->jump, h->phi, p, phi_corr, s));
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

gfm_status gfm_set_tuning(gfm_handle h, const gfm_tuning *t)
{
    if (!h || !t) return GFM_ERR_ARG;
    gfm_tuning nt = h->tuning;
    if (t->threads) nt.threads = t->threads;
    if (t->ctas_per_sm) nt.ctas_per_sm = t->ctas_per_sm;
    if (nt.threads < 32 || nt.threads > gfm::solver_max_threads() || nt.threads % 32 || nt.ctas_per_sm < 1)
        return fail(h, GFM_ERR_ARG, "threads must be a multiple of 32 in [32, 1024], ctas_per_sm >= 1");
    for (gfm::Mode m : {gfm::Mode::FP64, gfm::Mode::MIXED}) {
        int occ = 0;
        GFM_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gfm::solver_kernel(m, h->ht.max_width, nt.threads), nt.threads, 0));
        if (occ < nt.ctas_per_sm) return fail(h, GFM_ERR_ARG, "launch shape cannot be co-resident");
    }
    if (h->sm_count * nt.ctas_per_sm > h->max_grid) return fail(h, GFM_ERR_ARG, "grid larger than workspace");
    h->tuning = nt;
    return GFM_OK;
}

gfm_status gfm_get_tuning(gfm_handle h, gfm_tuning *t)
{
    if (!h || !t) return GFM_ERR_ARG;
    *t = h->tuning;
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
        cudaEventSynchronize(h->ev[5]);
        cudaEventElapsedTime(&h->prof.ms_assemble, h->ev[0], h->ev[1]);
        cudaEventElapsedTime(&h->prof.ms_solve, h->ev[2], h->ev[3]);
        cudaEventElapsedTime(&h->prof.ms_total, h->ev[4], h->ev[5]);
    }
    *out = h->prof;
    return GFM_OK;
}

gfm_status gfm_get_sizes(gfm_handle h, int32_t *n_cells, int32_t *n_faces, int32_t *n_tanks)
{
    if (!h) return GFM_ERR_ARG;
    if (n_cells) *n_cells = h->n;
    if (n_faces) *n_faces = h->F;
    if (n_tanks) *n_tanks = 1;
    return GFM_OK;
}

gfm_status gfm_get_permutation(gfm_handle h, int32_t *perm_host)
{
    if (!h || !perm_host) return GFM_ERR_ARG;
    std::memcpy(perm_host, h->ht.perm.data(), sizeof(int32_t) * (size_t)h->n);
    return GFM_OK;
}

}  // extern "C"
