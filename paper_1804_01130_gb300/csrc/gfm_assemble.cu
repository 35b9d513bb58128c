// Assembly of the Ghost Fluid Method pressure equation (Sec. 3.1, Eqs. 7,
// 12-20) and the per-face adjoint chain rule.
//
// This translation unit is compiled with --fmad=false: every FP64 expression
// rounds exactly as written, left to right, so the face quantities and the
// ordered per-cell sums are bit-reproducible against any IEEE-754 FP64
// evaluation of the same formulas in the same order.
#include "gfm_internal.h"

namespace gfm {

enum : int8_t { kDry = 0, kWet = 1, kIfOwnerWet = 2, kIfOwnerDry = 3 };

// One thread per internal face (caller order).
//   wet = alpha >= 0.5 (Sec. 3.1: the alpha = 0.5 contour is the interface;
//   alpha exactly 0.5 is taken as wet).
//   interface face: wet owner != wet neighbour.  W = wet cell, D = dry cell.
//   lambda = (alpha_W - 0.5) / (alpha_W - alpha_D)                 Eq. 13
//   c      = (S.S) / (S.d),  d = C_nb - C_own
//   gamma  = c / (lambda rho_w + (1 - lambda) rho_a)  = c beta+ beta- / beta_w   Eqs. 16-18, 20
//            (times the face Rhie-Chow coefficient rau_f when one is set)
//   x_G    = C_W + lambda (C_D - C_W)                              Eq. 12
//   H      = (rho_w - rho_a) g.x_G  = p_d(dry) - p_d(wet)           Eq. 7
//   J      = +H (owner wet) / -H (owner dry) / 0 (no interface)
//   sigma  = phi + gamma J   (the face's total source flux)
// Off the interface lambda is 1 (both wet) or 0 (both dry), which yields the
// phase density exactly.
__global__ void k_faces(FaceArgs a)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= a.F) return;
    const int o = a.owner[f], nb = a.neighbour[f];
    const size_t n = (size_t)a.n, F = (size_t)a.F;
    const double ao = a.alpha[o], an = a.alpha[nb];
    const bool wo = ao >= 0.5, wn = an >= 0.5;
    int8_t kind;
    double lam;
    int W = o, D = nb;
    if (wo == wn) {
        kind = wo ? kWet : kDry;
        lam = wo ? 1.0 : 0.0;
    } else {
        kind = wo ? kIfOwnerWet : kIfOwnerDry;
        if (!wo) { W = nb; D = o; }
        const double aW = a.alpha[W], aD = a.alpha[D];
        lam = (aW - 0.5) / (aW - aD);
    }
    double rho_w = a.rho_w, rho_a = a.rho_a, g0 = a.g0, g1 = a.g1, g2 = a.g2;
    if (a.ftank) {
        const TankPhys tp = a.tphys[a.ftank[f]];
        rho_w = tp.rho_w;
        rho_a = tp.rho_a;
        g0 = tp.g0;
        g1 = tp.g1;
        g2 = tp.g2;
    }
    const double Sx = a.Sf[f], Sy = a.Sf[F + f], Sz = a.Sf[2 * F + f];
    const double dx = a.C[nb] - a.C[o];
    const double dy = a.C[n + nb] - a.C[n + o];
    const double dz = a.C[2 * n + nb] - a.C[2 * n + o];
    const double c = (Sx * Sx + Sy * Sy + Sz * Sz) / (Sx * dx + Sy * dy + Sz * dz);
    const double rf = lam * rho_w + (1.0 - lam) * rho_a;
    double gam = c / rf;
    if (a.rau) gam = gam * a.rau[f];  // face Rhie-Chow coefficient 1/a_P
    double J = 0.0;
    if (kind >= kIfOwnerWet) {
        const double xg0 = a.C[W] + lam * (a.C[D] - a.C[W]);
        const double xg1 = a.C[n + W] + lam * (a.C[n + D] - a.C[n + W]);
        const double xg2 = a.C[2 * n + W] + lam * (a.C[2 * n + D] - a.C[2 * n + W]);
        const double H = (rho_w - rho_a) * ((g0 * xg0 + g1 * xg1) + g2 * xg2);
        J = (kind == kIfOwnerWet) ? H : -H;
    }
    a.lambda[f] = lam;
    a.gamma[f] = gam;
    a.jump[f] = J;
    a.sigma[f] = a.phi[f] + gam * J;
    a.kind[f] = kind;
}

// One thread per internal cell (lane l of slice s = cell 32 s + l).  Walks
// the cell's faces in ascending caller face order:
//   diag_i = sum gamma_f,  b_i = -sum s_if sigma_f  (s = +1 owner, -1 neighbour)
// fills the sliced-ELL coefficients (FP64 and FP32 copies), and applies the
// pin: b_r += diag_r * ref_value, diag_r += diag_r.
__global__ void k_cells(CellArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && !a.stank) a.prm->ref = a.ref;
    if (t >= a.m.n_pad) return;
    const int s = t >> 5, l = t & 31;
    int ref = a.ref;
    double ref_value = a.ref_value;
    DevParams *prm = a.prm;
    if (a.stank) {
        const int tk = a.stank[s];
        ref = a.tphys[tk].ref;
        ref_value = a.tphys[tk].ref_value;
        prm = a.tprm + tk;
    }
    const bool valid = a.iperm[t] >= 0;
    const int base = a.m.slice_ptr[s];
    const int w = (a.m.slice_ptr[s + 1] - base) >> 5;
    double diag = 0.0, b = 0.0;
    for (int k = 0; k < w; ++k) {
        const int slot = base + k * kSlice + l;
        const int code = a.m.face[slot];
        if (code == 0) {
            a.m.val64[slot] = 0.0;
            a.m.val32[slot] = 0.0f;
            if (a.ent) a.ent[slot] = (uint32_t)a.pad_code << 16;  // itself, coefficient 0
            continue;
        }
        const int f = (code > 0 ? code : -code) - 1;
        const double g = a.gamma[f];
        const double sg = a.sigma[f];
        diag = diag + g;
        b = (code > 0) ? b - sg : b + sg;
        a.m.val64[slot] = g;
        a.m.val32[slot] = (float)g;
        if (a.ent) {
            // off the interface the coefficient is the class's one for the
            // face's phase; interface faces read val32 (escape)
            const int8_t kd = a.kind[f];
            const uint32_t vc = kd == kWet ? (uint32_t)(2 * a.fcls[f]) : kd == kDry ? (uint32_t)(2 * a.fcls[f] + 1)
                                                                                  : kEscape;
            const int off = a.m.col[slot] - t;
            a.ent[slot] = (vc << 16) | ((uint32_t)off & 0xFFFFu);
        }
    }
    if (t == ref) {
        b = b + diag * ref_value;
        prm->pin64 = diag;
        prm->pin32 = (float)diag;
        diag = diag + diag;
    }
    a.b[t] = valid ? b : 0.0;
    a.diag[t] = valid ? diag : 0.0;
    a.dinv[t] = valid ? 1.0 / diag : 0.0;
    a.dinv32[t] = valid ? 1.0f / (float)diag : 0.0f;
}

// sigma = phi + gamma J for a new predicted flux on an assembled system (the
// interface, the coefficients and the jump unchanged), rounded as in k_faces.
__global__ void k_sigma(int F, const double *__restrict__ phi, const double *__restrict__ gamma,
                        const double *__restrict__ jump, double *__restrict__ sigma)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    sigma[f] = phi[f] + gamma[f] * jump[f];
}

// c_f = (S.S)/(S.d) per face, the geometric factor of gamma_f, rounded as in
// k_faces (the compact table groups faces of bit-identical c_f into classes).
__global__ void k_face_c(int n, int F, const int32_t *__restrict__ owner, const int32_t *__restrict__ neighbour,
                         const double *__restrict__ Sf, const double *__restrict__ C, double *__restrict__ out)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int o = owner[f], nb = neighbour[f];
    const size_t nn = (size_t)n, FF = (size_t)F;
    const double Sx = Sf[f], Sy = Sf[FF + f], Sz = Sf[2 * FF + f];
    const double dx = C[nb] - C[o];
    const double dy = C[nn + nb] - C[nn + o];
    const double dz = C[2 * nn + nb] - C[2 * nn + o];
    out[f] = (Sx * Sx + Sy * Sy + Sz * Sz) / (Sx * dx + Sy * dy + Sz * dz);
}

// Dictionary of the compact table: the off-interface coefficients
// c / (lambda rho_w + (1 - lambda) rho_a) with lambda = 1 (wet) and 0 (dry),
// written with k_faces' expression so each entry has the bits of the
// gamma_f (as FP32) of the faces it stands for.
__global__ void k_dict(DictArgs a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) a.dict[2 * a.n_cls] = 0.0f;  // padding slots
    if (k >= a.n_cls) return;
    double rho_w = a.rho_w, rho_a = a.rho_a;
    if (a.ctank) {
        const TankPhys tp = a.tphys[a.ctank[k]];
        rho_w = tp.rho_w;
        rho_a = tp.rho_a;
    }
    const double c = a.ccls[k];
    const double lw = 1.0, ld = 0.0;
    const double rfw = lw * rho_w + (1.0 - lw) * rho_a;
    const double rfd = ld * rho_w + (1.0 - ld) * rho_a;
    a.dict[2 * k] = (float)(c / rfw);
    a.dict[2 * k + 1] = (float)(c / rfd);
}

// sum(b) and sum(|b|) by one block, fixed order (compatibility check of an
// unpinned system).
__global__ void k_bsums(const double *__restrict__ b, int n, DevParams *prm)
{
    __shared__ double s1[32], s2[32];
    double a1 = 0.0, a2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a1 += b[i];
        a2 += fabs(b[i]);
    }
    for (int off = 16; off; off >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    }
    if ((threadIdx.x & 31) == 0) { s1[threadIdx.x >> 5] = a1; s2[threadIdx.x >> 5] = a2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { t1 += s1[k]; t2 += s2[k]; }
        prm->bsum = t1;
        prm->babs = t2;
    }
}

// Corrected face flux phi_f = phi*_f - gamma_f (p_nb - p_own - J_f).
__global__ void k_corrected_flux(int F, const int32_t *__restrict__ owner, const int32_t *__restrict__ nb,
                                 const double *__restrict__ gamma, const double *__restrict__ jump,
                                 const double *__restrict__ phi, const double *__restrict__ p,
                                 double *__restrict__ out)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const int o = owner[f], n = nb[f];
    out[f] = phi[f] - gamma[f] * ((p[n] - p[o]) - jump[f]);
}

// Adjoint, per face (caller order).  With mu = A^{-1} dL/dp:
//   dL/dphi_f   = -(mu_o - mu_nb)
//   dL/dgamma_f = -(mu_o - mu_nb)(p_o - p_nb + J_f),  dL/dJ_f = -gamma_f (mu_o - mu_nb)
//   dgamma/dlambda = -gamma (rho_w - rho_a)/rho_f,  dJ/dlambda = +-(rho_w - rho_a) g.(x_D - x_W)
//   dL/dlambda_f = dL/dgamma dgamma/dlambda + dL/dJ dJ/dlambda  (interface faces; 0 elsewhere)
__global__ void k_adjoint_faces(AdjointArgs a)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= a.F) return;
    const int o = a.owner[f], nb = a.neighbour[f];
    const size_t n = (size_t)a.n;
    const double dmu = a.mu[o] - a.mu[nb];
    a.dL_dphi[f] = -dmu;
    double dlam = 0.0;
    const int8_t kind = a.kind[f];
    if (kind >= kIfOwnerWet) {
        const int W = (kind == kIfOwnerWet) ? o : nb;
        const int D = (kind == kIfOwnerWet) ? nb : o;
        const double lam = a.lambda[f];
        const double gam = a.gamma[f];
        const double rf = lam * a.rho_w + (1.0 - lam) * a.rho_a;
        const double dgam_dlam = -gam * (a.rho_w - a.rho_a) / rf;
        double gd = 0.0;
        gd += a.g0 * (a.C[D] - a.C[W]);
        gd += a.g1 * (a.C[n + D] - a.C[n + W]);
        gd += a.g2 * (a.C[2 * n + D] - a.C[2 * n + W]);
        const double dH_dlam = (a.rho_w - a.rho_a) * gd;
        const double dJ_dlam = (kind == kIfOwnerWet) ? dH_dlam : -dH_dlam;
        const double dL_dgam = -dmu * ((a.p[o] - a.p[nb]) + a.jump[f]);
        const double dL_dJ = -gam * dmu;
        dlam = dL_dgam * dgam_dlam + dL_dJ * dJ_dlam;
    }
    a.dL_dlam[f] = dlam;
}

// Adjoint, per cell (internal order, faces in ascending caller order):
//   dL/dalpha_i = sum over interface faces f of i of dL/dlambda_f dlambda_f/dalpha_i,
//   dlambda/dalpha_W = (0.5 - alpha_D)/(alpha_W - alpha_D)^2,
//   dlambda/dalpha_D = (alpha_W - 0.5)/(alpha_W - alpha_D)^2          (from Eq. 13)
__global__ void k_adjoint_cells(AdjointArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.m.n) return;
    const int s = t >> 5, l = t & 31;
    const int base = a.m.slice_ptr[s];
    const int w = (a.m.slice_ptr[s + 1] - base) >> 5;
    const int me = a.iperm[t];
    double acc = 0.0;
    for (int k = 0; k < w; ++k) {
        const int code = a.m.face[base + k * kSlice + l];
        if (code == 0) continue;
        const int f = (code > 0 ? code : -code) - 1;
        const int8_t kind = a.kind[f];
        if (kind < kIfOwnerWet) continue;
        const int o = a.owner[f], nb = a.neighbour[f];
        const int W = (kind == kIfOwnerWet) ? o : nb;
        const int D = (kind == kIfOwnerWet) ? nb : o;
        const double aW = a.alpha[W], aD = a.alpha[D];
        const double den = (aW - aD) * (aW - aD);
        const double d = (me == W) ? (0.5 - aD) / den : (aW - 0.5) / den;
        acc += a.dL_dlam[f] * d;
    }
    a.dL_dalpha[me] = acc;
}

// dst[i] = src[iperm[i]] (caller order -> internal order), zero on padding
// cells (iperm = -1).
__global__ void k_gather(const double *__restrict__ src, const int32_t *__restrict__ iperm, double *__restrict__ dst,
                         int n, int n_pad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const int c = iperm[i];
    dst[i] = (c >= 0) ? src[c] : 0.0;
}

static inline int blocks_for(long long work, int threads) { return (int)((work + threads - 1) / threads); }

cudaError_t launch_faces(const FaceArgs &a, cudaStream_t s)
{
    if (a.F <= 0) return cudaSuccess;
    k_faces<<<blocks_for(a.F, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cells(const CellArgs &a, cudaStream_t s)
{
    k_cells<<<blocks_for(a.m.n_pad, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bsums(const double *b, int32_t n, DevParams *prm, cudaStream_t s)
{
    k_bsums<<<1, 1024, 0, s>>>(b, n, prm);
    return cudaGetLastError();
}

cudaError_t launch_face_c(int32_t n, int32_t F, const int32_t *owner, const int32_t *neighbour, const double *Sf,
                          const double *C, double *c, cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    k_face_c<<<blocks_for(F, 256), 256, 0, s>>>(n, F, owner, neighbour, Sf, C, c);
    return cudaGetLastError();
}

cudaError_t launch_sigma(int32_t F, const double *phi, const double *gamma, const double *jump, double *sigma,
                         cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    k_sigma<<<blocks_for(F, 256), 256, 0, s>>>(F, phi, gamma, jump, sigma);
    return cudaGetLastError();
}

cudaError_t launch_dict(const DictArgs &a, cudaStream_t s)
{
    k_dict<<<blocks_for(a.n_cls + 1, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_corrected_flux(int32_t F, const int32_t *owner, const int32_t *neighbour, const double *gamma,
                                  const double *jump, const double *phi, const double *p, double *out,
                                  cudaStream_t s)
{
    if (F <= 0) return cudaSuccess;
    k_corrected_flux<<<blocks_for(F, 256), 256, 0, s>>>(F, owner, neighbour, gamma, jump, phi, p, out);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_faces(const AdjointArgs &a, cudaStream_t s)
{
    k_adjoint_faces<<<blocks_for(a.F, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_cells(const AdjointArgs &a, cudaStream_t s)
{
    k_adjoint_cells<<<blocks_for(a.m.n, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gather(const double *src_user, const int32_t *iperm, double *dst_internal, int32_t n,
                          int32_t n_pad, cudaStream_t s)
{
    k_gather<<<blocks_for(n_pad, 256), 256, 0, s>>>(src_user, iperm, dst_internal, n, n_pad);
    return cudaGetLastError();
}

}  // namespace gfm
