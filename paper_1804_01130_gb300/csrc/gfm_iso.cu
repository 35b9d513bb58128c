// isoAdvector advection step (Sec. 3.2): the heavy-fluid volume each face
// passes during a time step, and the volume-fraction update.
//
// Over [t, t + dt] the face passes dV_f = phi_f int alpha_f+(tau) dtau
// (Eq. dV), alpha_f+ being the submerged fraction of the face (Eq. alphaf).
// In the upwind cell the interface is the isoface plane (centre x_S, unit
// normal n_S away from the heavy fluid) moving at normal speed U_S.n_S, so a
// point x is reached at t_x = (x - x_S).n_S / U_S.n_S (Eq. tv).  The face is
// the union of triangles (face centre, v_k, v_k+1).  On each triangle with
// vertex times t1 <= t2 <= t3 the sweep line enters at x1, passes x2 while
// cutting edge 1-3 at x4 (Eq. x_41), and leaves at x3; the swept fraction is
// quadratic in tau on [t1, t2] and on [t2, t3] (Eqs. aplus1, aplus2) with
//     a2 = |x41 x x21| / 2A        (the swept fraction at t2),
//     F  = a2 ((tau - t1)/(t2 - t1))^2              on [t1, t2],
//     F  = 1 - (1 - a2) ((t3 - tau)/(t3 - t2))^2    on [t2, t3],
// and the time integral over [0, dt] is the sum of the pieces' exact
// integrals (Eq. intaplus), written in shifted form for conditioning.  When
// the interface moves towards the heavy fluid (U_S.n_S < 0) the swept part
// is the part that has drained: the submerged fraction is 1 - F.  A face
// whose upwind cell has no isoface carries that cell's alpha throughout.
//
// One thread per face (FP64 geometry); then one thread per cell sums its
// faces' volumes in ascending face order through the sliced-ELL table:
//     alpha_P(t + dt) = alpha_P(t) - 1/V_P sum_f s_Pf dV_f.
#include "gfm_internal.h"

namespace gfm {

namespace {

struct V3 {
    double x, y, z;
};

__device__ __forceinline__ V3 sub(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double cross_norm(V3 a, V3 b)
{
    const double cx = a.y * b.z - a.z * b.y, cy = a.z * b.x - a.x * b.z, cz = a.x * b.y - a.y * b.x;
    return sqrt(cx * cx + cy * cy + cz * cz);
}

// The sweep of one triangle: vertex times in order and the swept fraction
// a2 at the middle time.
struct Sweep {
    double t1, t2, t3, a2;
};

__device__ Sweep make_sweep(V3 x1, V3 x2, V3 x3, double t1, double t2, double t3)
{
    // order the vertices by arrival time
    if (t1 > t2) { const double q = t1; t1 = t2; t2 = q; const V3 r = x1; x1 = x2; x2 = r; }
    if (t2 > t3) { const double q = t2; t2 = t3; t3 = q; const V3 r = x2; x2 = x3; x3 = r; }
    if (t1 > t2) { const double q = t1; t1 = t2; t2 = q; const V3 r = x1; x1 = x2; x2 = r; }
    const V3 x21 = sub(x2, x1), x31 = sub(x3, x1);
    const double A2 = cross_norm(x31, x21);  // twice the triangle's area
    // x4 on edge 1-3, reached at t2: x41 = ((t2 - t1)/(t3 - t1)) x31 (Eq. x_41)
    double a2 = 1.0;
    if (t3 > t1 && A2 > 0.0) {
        const double r = (t2 - t1) / (t3 - t1);
        a2 = cross_norm(V3{r * x31.x, r * x31.y, r * x31.z}, x21) / A2;
    }
    return Sweep{t1, t2, t3, a2};
}

// The swept fraction F(tau) (Eqs. aplus1, aplus2).
__device__ double sweep_at(const Sweep &w, double tau)
{
    if (tau <= w.t1) return 0.0;
    if (tau <= w.t2) {
        const double q = (tau - w.t1) / (w.t2 - w.t1);
        return w.a2 * q * q;
    }
    if (tau < w.t3) {
        const double q = (w.t3 - tau) / (w.t3 - w.t2);
        return 1.0 - (1.0 - w.a2) * q * q;
    }
    return 1.0;
}

// int_0^dt F(tau) dtau: the exact integrals of the quadratic pieces clipped
// to [0, dt] (Eq. intaplus, in shifted form).
__device__ double sweep_integral(const Sweep &w, double dt)
{
    double I = 0.0;
    if (w.t2 > w.t1) {  // [t1, t2]: a2 ((tau - t1)/(t2 - t1))^2
        const double lo = fmin(fmax(0.0, w.t1), w.t2), hi = fmin(fmax(dt, w.t1), w.t2);
        if (hi > lo) {
            const double d = w.t2 - w.t1, u = hi - w.t1, l = lo - w.t1;
            I += w.a2 * (u * u * u - l * l * l) / (3.0 * d * d);
        }
    }
    if (w.t3 > w.t2) {  // [t2, t3]: 1 - (1 - a2) ((t3 - tau)/(t3 - t2))^2
        const double lo = fmin(fmax(0.0, w.t2), w.t3), hi = fmin(fmax(dt, w.t2), w.t3);
        if (hi > lo) {
            const double d = w.t3 - w.t2, u = w.t3 - lo, l = w.t3 - hi;
            I += (hi - lo) - (1.0 - w.a2) * (u * u * u - l * l * l) / (3.0 * d * d);
        }
    }
    const double s3 = fmax(0.0, w.t3);  // [t3, dt]: fully swept
    if (dt > s3) I += dt - s3;
    return I;
}

__global__ void __launch_bounds__(256) k_iso_flux(IsoArgs a)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= a.F) return;
    const size_t n = (size_t)a.n, F = (size_t)a.F, nvt = (size_t)a.nvt;
    const double ph = a.phi[f];
    const int U = ph >= 0.0 ? a.owner[f] : a.neighbour[f];
    double I;
    if (!a.has_iso[U]) {
        I = a.alpha[U] * a.dt;
    } else {
        const V3 xs{a.xS[U], a.xS[n + U], a.xS[2 * n + U]};
        const V3 ns{a.nS[U], a.nS[n + U], a.nS[2 * n + U]};
        const double un = a.UnS[U];
        const V3 c{a.xf[f], a.xf[F + f], a.xf[2 * F + f]};
        const int v0 = a.fv_ptr[f], nv = a.fv_ptr[f + 1] - v0;
        // a static interface (U_S.n_S = 0): the fraction behind the plane,
        // the sweep read at tau = 0 with the signed distances as times
        const bool moving = un != 0.0;
        const double iu = moving ? 1.0 / un : 1.0;
        double atot = 0.0, acc = 0.0;
        V3 pa{a.fv_xyz[v0], a.fv_xyz[nvt + v0], a.fv_xyz[2 * nvt + v0]};
        for (int e = 0; e < nv; ++e) {
            const int q = v0 + (e + 1 < nv ? e + 1 : 0);
            const V3 pb{a.fv_xyz[q], a.fv_xyz[nvt + q], a.fv_xyz[2 * nvt + q]};
            const double at = cross_norm(sub(pa, c), sub(pb, c));  // twice the area
            if (at > 0.0) {
                const Sweep w = make_sweep(c, pa, pb, dot(sub(c, xs), ns) * iu, dot(sub(pa, xs), ns) * iu,
                                           dot(sub(pb, xs), ns) * iu);
                double sw;
                if (!moving) sw = sweep_at(w, 0.0) * a.dt;
                else {
                    sw = sweep_integral(w, a.dt);
                    if (un < 0.0) sw = a.dt - sw;  // moving into the heavy fluid: the swept part has drained
                }
                atot += at;
                acc += at * sw;
            }
            pa = pb;
        }
        I = atot > 0.0 ? acc / atot : 0.0;
    }
    if (a.integral) a.integral[f] = I;
    a.dV[f] = ph * I;
}

__global__ void __launch_bounds__(256) k_iso_cells(IsoArgs a)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.m.n_pad) return;
    const int c = a.iperm[t];
    if (c < 0) return;
    const int s = t / kSlice, l = t % kSlice;
    const int base = a.m.slice_ptr[s];
    const int w = (a.m.slice_ptr[s + 1] - base) / kSlice;
    double acc = 0.0;
    for (int k = 0; k < w; ++k) {
        const int code = a.m.face[base + k * kSlice + l];
        if (code == 0) continue;
        const int f = (code > 0 ? code : -code) - 1;
        acc = (code > 0) ? acc + a.dV[f] : acc - a.dV[f];
    }
    a.alpha_new[c] = a.alpha[c] - acc / a.V[c];
}

}  // namespace

cudaError_t launch_iso(const IsoArgs &a, cudaStream_t s)
{
    if (a.F > 0) k_iso_flux<<<(a.F + 255) / 256, 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !a.alpha_new) return e;
    k_iso_cells<<<(a.m.n_pad + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gfm
