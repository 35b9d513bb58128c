// Dynamic-pressure gradient of the momentum equation and cell velocities
// from face fluxes (Sec. 3.1, Eq. 20 and the paragraph after it; Eq. 2's
// pressure term, Eq. 8).
//
// The momentum equation needs (1/rho) grad p_d at cell centres.  By the
// Gauss theorem with linear cell-to-face interpolation, cell P sees face f
// through p_f = w_P p_P + (1 - w_P) pN~, where pN~ is the neighbour's value,
// replaced at an interface face by its ghost value extrapolated into P's
// fluid (Eq. 20 from the wet side, the analogous expression from the dry
// side).  Written out, both ghost values collapse onto the coefficients the
// assembly already holds:
//     beta_P (pN~ - p_P) = (p_N - p_P - s_Pf J_f) / rho_f,
//     rho_f = lambda_f rho_w + (1 - lambda_f) rho_a   (the harmonic face density of Eq. 18),
// J_f the oriented jump (Eq. 7) and s_Pf = +1 if P owns f, -1 otherwise; off
// the interface J_f = 0 and rho_f is the phase's own density.  With
// zero-gradient walls the face sum reduces to the internal faces in
// difference form, so
//     (1/rho grad p_d)_P = 1/V_P sum_f (1 - w_P) (p_N - p_P - s_Pf J_f) / rho_f  s_Pf S_f,
//     (1 - w_P) = S_f.(x_f - x_P) / S_f.(x_N - x_P).
// The reconstruction of a cell velocity from face fluxes uses the identity
// sum_f (u.S_f)(x_f - x_P) = V_P u of a closed cell:
//     U_P = 1/V_P sum_f s_Pf phi_f (x_f - x_P).
//
// One thread per cell walks the cell's faces in the sliced-ELL table
// (ascending face order) and gathers the neighbour's p_d and centre; face
// arrays are read in the caller's face order.  FP64 throughout.
#include "gfm_internal.h"

namespace gfm {

namespace {

__global__ void __launch_bounds__(256) k_gradient(GradArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m.n_pad) return;
    const int c = a.iperm[i];
    if (c < 0) return;  // padding cell
    const int s = i / kSlice, lane = i % kSlice;
    const int base = a.m.slice_ptr[s];
    const int w = (a.m.slice_ptr[s + 1] - base) / kSlice;
    double rho_w = a.rho_w, rho_a = a.rho_a;
    if (a.stank) {
        const TankPhys tp = a.tphys[a.stank[s]];
        rho_w = tp.rho_w;
        rho_a = tp.rho_a;
    }
    const int n = a.n, F = a.F;
    const double pP = a.p[c];
    const double xP0 = a.C[c], xP1 = a.C[(size_t)n + c], xP2 = a.C[2 * (size_t)n + c];
    double g0 = 0.0, g1 = 0.0, g2 = 0.0, u0 = 0.0, u1 = 0.0, u2 = 0.0;
    for (int k = 0; k < w; ++k) {
        const int fo = a.m.face[base + k * kSlice + lane];
        if (fo == 0) continue;  // padding slot
        const int f = (fo > 0 ? fo : -fo) - 1;
        const double sg = fo > 0 ? 1.0 : -1.0;
        const int cN = fo > 0 ? a.neighbour[f] : a.owner[f];
        const double S0 = a.Sf[f], S1 = a.Sf[(size_t)F + f], S2 = a.Sf[2 * (size_t)F + f];
        const double dN0 = a.C[cN] - xP0, dN1 = a.C[(size_t)n + cN] - xP1, dN2 = a.C[2 * (size_t)n + cN] - xP2;
        double df0, df1, df2;  // x_f - x_P
        if (a.xf) {
            df0 = a.xf[f] - xP0;
            df1 = a.xf[(size_t)F + f] - xP1;
            df2 = a.xf[2 * (size_t)F + f] - xP2;
        } else {  // face centre half-way between the cell centres
            df0 = 0.5 * dN0;
            df1 = 0.5 * dN1;
            df2 = 0.5 * dN2;
        }
        if (a.grad) {
            const double lam = a.lambda[f];
            const double rf = lam * rho_w + (1.0 - lam) * rho_a;
            const double delta = (a.p[cN] - pP) - sg * a.jump[f];
            const double fac = a.xf ? (S0 * df0 + S1 * df1 + S2 * df2) / (S0 * dN0 + S1 * dN1 + S2 * dN2) : 0.5;
            const double cf = sg * fac * delta / rf;
            g0 += cf * S0;
            g1 += cf * S1;
            g2 += cf * S2;
        }
        if (a.U) {
            const double ph = sg * a.phi[f];
            u0 += ph * df0;
            u1 += ph * df1;
            u2 += ph * df2;
        }
    }
    const double iv = 1.0 / a.V[c];
    if (a.grad) {
        a.grad[c] = g0 * iv;
        a.grad[(size_t)n + c] = g1 * iv;
        a.grad[2 * (size_t)n + c] = g2 * iv;
    }
    if (a.U) {
        a.U[c] = u0 * iv;
        a.U[(size_t)n + c] = u1 * iv;
        a.U[2 * (size_t)n + c] = u2 * iv;
    }
}

// Explicit over-relaxed non-orthogonal correction (Sec. 3), one thread per
// face: S_f = Delta_f + k_f with Delta_f = (S.S)/(S.d) d along the centre
// line (the implicit two-point part), and the k part from the gradient of
// the last p_d, interpolated to the face with the face-centre weight:
//     corr_f = rau_f k_f . (w_o G_own + (1 - w_o) G_nb),
// G = (1/rho) grad p_d (continuous across the interface by Eq. 8).  The face
// flux then reads phi*_f - corr_f - gamma_f (p_nb - p_own - J_f), so the cell
// sums take phi_eff = phi* - corr and sigma = phi_eff + gamma J.
__global__ void __launch_bounds__(256) k_nonorth(NonorthArgs a)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= a.F) return;
    const size_t n = (size_t)a.n, F = (size_t)a.F;
    const int o = a.owner[f], nb = a.neighbour[f];
    double S[3], d[3], x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        S[k] = a.Sf[k * F + f];
        d[k] = a.C[k * n + nb] - a.C[k * n + o];
        x[k] = a.xf ? a.xf[k * F + f] : 0.5 * (a.C[k * n + o] + a.C[k * n + nb]);
    }
    const double ss = S[0] * S[0] + S[1] * S[1] + S[2] * S[2];
    const double sd = S[0] * d[0] + S[1] * d[1] + S[2] * d[2];
    double snf = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) snf += S[k] * (a.C[k * n + nb] - x[k]);
    const double w_o = snf / sd;
    double kg = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double kf = S[k] - (ss / sd) * d[k];
        const double Gf = w_o * a.G[k * n + o] + (1.0 - w_o) * a.G[k * n + nb];
        kg += kf * Gf;
    }
    const double corr = (a.rau ? a.rau[f] : 1.0) * kg;
    const double pe = a.phi[f] - corr;
    a.corr[f] = corr;
    a.phi_eff[f] = pe;
    a.sigma[f] = pe + a.gamma[f] * a.jump[f];
}

}  // namespace

cudaError_t launch_nonorth(const NonorthArgs &a, cudaStream_t s)
{
    if (a.F <= 0) return cudaSuccess;
    k_nonorth<<<(a.F + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gradient(const GradArgs &a, cudaStream_t s)
{
    if (a.m.n_pad <= 0) return cudaSuccess;
    k_gradient<<<(a.m.n_pad + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gfm
