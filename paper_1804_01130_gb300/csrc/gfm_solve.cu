// Persistent, cooperative solver kernels for the GFM pressure equation.
//
// The paper names no linear solver (it reports residual levels only,
// Sec. 4.1.1); both kernels run Jacobi-preconditioned conjugate gradients on
// the symmetric positive definite pinned system of Sec. 3.1.
//
//  k_solve_fp64  : textbook PCG, all FP64, three passes per iteration
//                  (SpMV + p.q | x, r update + preconditioner + r.z | new
//                  direction) separated by grid barriers.  On GB300 FP64 runs
//                  at 2 FMA/clk/SM, so this path keeps its FP64 operations
//                  per cell to the minimum (diagonal-form SpMV, stored 1/diag).
//  k_solve_mixed : FP32 PCG with FP64 "reliable updates" (residual
//                  replacement): the FP64 solution x, the true residual
//                  b - A x and the jump source never leave FP64.  Each FP32
//                  iteration is two passes and two grid barriers: (A) the new
//                  direction p = u + beta p is formed for the cell and,
//                  redundantly, for its neighbours from the gathered (u, p)
//                  pair, then s = A p and p.s; (B) e += alpha p,
//                  r -= alpha s, u = D^{-1} r, r.u and r.r.  Whenever the
//                  FP32 residual has dropped by a decade since the last
//                  replacement (or claims convergence), e is folded into x in
//                  FP64 and r is replaced by the true FP64 residual; the
//                  search direction is kept, so the Krylov space is not
//                  thrown away.  Dot products: FP32 products summed in
//                  double-float (TwoSum) per thread, warp and CTA, then FP64
//                  across CTAs, so no per-cell FP64 instruction runs in the
//                  FP32 iterations.
//
// All scalar recurrences (alpha, beta, stopping tests) run in ONE thread per
// CTA and are broadcast through shared memory: on GB300 the FP64 pipe is 1/64
// of the FP32 rate, and a scalar FP64 divide repeated by every thread cost
// more than the pass it controls.
//
// The FP32 operator is applied in difference form, (A p)_i = sum_f gamma_f
// (p_i - p_j) + pin_i p_i, which keeps the zero row sums of the GFM
// Laplacian exact and makes the FP32 operator spectrally equivalent to the
// FP64 one within one rounding of each gamma_f.
//
// Every row walk loads its slots' (neighbour, coefficient) pairs for a chunk
// of CH faces first and then issues all neighbour gathers together, so a row
// costs two dependent memory round trips instead of two per face.
//
// Grid barriers: one arrival counter, release-add / acquire-spin, every wait
// bounded by a globaltimer budget; on expiry the kernel records
// GFM_ERR_TIMEOUT and every CTA returns.  Reductions are deterministic: each
// CTA writes its partial sums, and after the barrier every CTA sums all
// partials in the same fixed order, so all CTAs take identical decisions.
#include "gfm_internal.h"

namespace gfm {

namespace {

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(const volatile int *)p; }

constexpr int kMaxNR = 6;

// Values decided by thread 0 and broadcast to the CTA.
struct Ctl {
    double alpha, beta, xavg;
    float al, be;
    int action;
};

struct Shared {
    float2 warp_ff[32][kMaxNR];
    double warp_d[32][kMaxNR];
    double out[kMaxNR];
    Ctl ctl;
    int flag;
};

struct Grid {
    unsigned *bar;
    int *err;
    double *partials;  // [2][kMaxNR][G]
    unsigned long long budget;
    unsigned epoch;
    int G;
    int parity;
};

// Grid-wide barrier.  Returns false if the solve must stop (a timeout here or
// an error recorded by any CTA).
__device__ bool grid_sync(Grid &g, Shared &sh)
{
    __syncthreads();
    g.epoch += 1u;
    if (threadIdx.x == 0) {
        int fail = 0;
        red_release_add_u32(g.bar, 1u);
        const unsigned target = g.epoch * (unsigned)g.G;
        const unsigned long long t0 = gtime();
        for (;;) {
            const unsigned v = ld_acquire_u32(g.bar);
            if ((int)(v - target) >= 0) break;
            if (ld_volatile_i32(g.err) != 0) { fail = 1; break; }
            if (gtime() - t0 > g.budget) {
                atomicCAS(g.err, 0, (int)GFM_ERR_TIMEOUT);
                fail = 1;
                break;
            }
        }
        __threadfence();
        if (!fail && ld_volatile_i32(g.err) != 0) fail = 1;
        sh.flag = fail;
    }
    __syncthreads();
    return sh.flag == 0;
}

// Deterministic all-reduce of NR doubles.  `blk` must hold this CTA's partial
// sums in thread 0.  Warp k sums value k over all CTAs (lane l takes CTAs
// l, l+32, ...; then a butterfly), identically in every CTA.
template <int NR>
__device__ bool grid_allreduce(Grid &g, Shared &sh, const double (&blk)[NR], double (&out)[NR])
{
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) g.partials[((size_t)g.parity * kMaxNR + k) * g.G + blockIdx.x] = blk[k];
    }
    if (!grid_sync(g, sh)) return false;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < NR) {
        const double *src = g.partials + ((size_t)g.parity * kMaxNR + warp) * g.G;
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int b = lane + 32 * q;
            v[q] = (b < g.G) ? __ldcg(src + b) : 0.0;
        }
        double acc = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        for (int b = lane + 256; b < g.G; b += 32) acc += __ldcg(src + b);
#pragma unroll
        for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) sh.out[warp] = acc;
    }
    g.parity ^= 1;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NR; ++k) out[k] = sh.out[k];
    return true;
}

// Block reduction of per-thread FP64 partials into thread 0 (fixed order).
template <int NR>
__device__ void block_sum_f64(Shared &sh, double (&v)[NR])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
#pragma unroll
        for (int off = 16; off; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) sh.warp_d[warp][k] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            double a = (lane < nw) ? sh.warp_d[lane][k] : 0.0;
#pragma unroll
            for (int off = 16; off; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            v[k] = a;
        }
    }
}

// Double-float accumulator: value = hi + lo, TwoSum updates (Knuth), so a
// long FP32 sum keeps ~48 bits.  Built from FP32 adds only.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ void ff_add(FF &a, float x)
{
    const float s = a.hi + x;
    const float bp = s - a.hi;
    const float e = (a.hi - (s - bp)) + (x - bp);
    a.hi = s;
    a.lo += e;
}

__device__ __forceinline__ FF ff_merge(FF a, FF b)
{
    const float s = a.hi + b.hi;
    const float bp = s - a.hi;
    float e = (a.hi - (s - bp)) + (b.hi - bp);
    e += a.lo + b.lo;
    const float hi = s + e;
    return FF{hi, e - (hi - s)};
}

__device__ __forceinline__ FF ff_shfl_tree(FF v)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        FF o;
        o.hi = __shfl_xor_sync(0xffffffffu, v.hi, off);
        o.lo = __shfl_xor_sync(0xffffffffu, v.lo, off);
        v = ff_merge(v, o);
    }
    return v;
}

// Block reduction of per-thread double-float partials; result (FP64) in
// thread 0.  Warps and the block both reduce in double-float.
template <int NR>
__device__ void block_sum_ff(Shared &sh, FF (&v)[NR], double (&out)[NR])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] = ff_shfl_tree(v[k]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) sh.warp_ff[warp][k] = make_float2(v[k].hi, v[k].lo);
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const float2 t = (lane < nw) ? sh.warp_ff[lane][k] : make_float2(0.f, 0.f);
            const FF r = ff_shfl_tree(FF{t.x, t.y});
            out[k] = (double)r.hi + (double)r.lo;
        }
    }
}

struct Range {
    int s0, s1, warp, lane, nw;
};

__device__ __forceinline__ Range my_range(int n_slices)
{
    Range r;
    const long long G = gridDim.x;
    r.s0 = (int)(((long long)n_slices * blockIdx.x) / G);
    r.s1 = (int)(((long long)n_slices * (blockIdx.x + 1)) / G);
    r.warp = threadIdx.x >> 5;
    r.lane = threadIdx.x & 31;
    r.nw = blockDim.x >> 5;
    return r;
}

struct Row {
    int base, w;
};

__device__ __forceinline__ Row row_of(const Sell &m, int s)
{
    const int base = __ldg(m.slice_ptr + s);
    return Row{base, (__ldg(m.slice_ptr + s + 1) - base) >> 5};
}

// (A x)_i in FP64, difference form: sum_f gamma_f (x_i - x_j) + pin x_i.
template <int CH>
__device__ __forceinline__ double apply64_diff(const Sell &m, Row rw, int lane, const double *x, double xi,
                                               double pin_i)
{
    double acc = pin_i * xi;
    for (int k0 = 0; k0 < rw.w; k0 += CH) {
        int j[CH];
        double gm[CH], xj[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const bool ok = k0 + c < rw.w;
            const int slot = rw.base + (k0 + c) * kSlice + lane;
            j[c] = ok ? __ldg(m.col + slot) : 0;
            gm[c] = ok ? __ldg(m.val64 + slot) : 0.0;
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) xj[c] = (k0 + c < rw.w) ? x[j[c]] : xi;
#pragma unroll
        for (int c = 0; c < CH; ++c) acc = fma(gm[c], xi - xj[c], acc);
    }
    return acc;
}

// (A x)_i in FP64, diagonal form: diag_i x_i - sum_f gamma_f x_j.
template <int CH>
__device__ __forceinline__ double apply64_diag(const Sell &m, Row rw, int lane, const double *x, double xi,
                                               double di)
{
    double acc = di * xi;
    for (int k0 = 0; k0 < rw.w; k0 += CH) {
        int j[CH];
        double gm[CH], xj[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const bool ok = k0 + c < rw.w;
            const int slot = rw.base + (k0 + c) * kSlice + lane;
            j[c] = ok ? __ldg(m.col + slot) : 0;
            gm[c] = ok ? __ldg(m.val64 + slot) : 0.0;
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) xj[c] = (k0 + c < rw.w) ? x[j[c]] : 0.0;
#pragma unroll
        for (int c = 0; c < CH; ++c) acc = fma(-gm[c], xj[c], acc);
    }
    return acc;
}

// FP32 diagonal D_i = pin_i + sum_f (float)gamma_f, summed in slot order.
__device__ __forceinline__ float diag32(const Sell &m, Row rw, int lane, float pin_i)
{
    float d = pin_i;
    for (int k = 0; k < rw.w; ++k) d += __ldg(m.val32 + rw.base + k * kSlice + lane);
    return d;
}

// Final two passes shared by both kernels: the true FP64 residual (difference
// form), the solution written in caller order, the OpenFOAM-style normalised
// L1 residual sum|r| / (sum|A x - x_avg rowsum| + sum|b - x_avg rowsum|),
// and the result record.  bnorm is only meaningful in thread 0.
template <int CH>
__device__ void finish(const SolveArgs &a, Grid &g, Shared &sh, const Range &R, int iters, int refinements,
                       int status, double bnorm)
{
    const int n = a.m.n;
    const int ref = a.prm->ref;
    const double pin = a.prm->pin64;
    if (!grid_sync(g, sh)) return;
    double v[2] = {0.0, 0.0};
    for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
        const int i = s * kSlice + R.lane;
        if (i < n) {
            const double xi = a.x64[i];
            const double r = a.b[i] - apply64_diff<CH>(a.m, row_of(a.m, s), R.lane, a.x64, xi, i == ref ? pin : 0.0);
            a.r64[i] = r;
            v[0] += r * r;
            v[1] += xi;
        }
    }
    block_sum_f64<2>(sh, v);
    double tot[2];
    if (!grid_allreduce<2>(g, sh, v, tot)) return;
    if (threadIdx.x == 0) sh.ctl.xavg = tot[1] / (double)n;
    __syncthreads();
    const double xavg = sh.ctl.xavg;
    double w[2] = {0.0, 0.0};
    for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
        const int i = s * kSlice + R.lane;
        if (i < n) {
            const double xi = a.x64[i];
            a.p_user[a.iperm[i]] = xi;
            const double r = a.r64[i];
            const double rs = (i == ref) ? pin : 0.0;
            const double Ax = a.b[i] - r;
            w[0] += fabs(r);
            w[1] += fabs(Ax - xavg * rs) + fabs(a.b[i] - xavg * rs);
        }
    }
    block_sum_f64<2>(sh, w);
    double l1[2];
    if (!grid_allreduce<2>(g, sh, w, l1)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int st = status;
        const int e = ld_volatile_i32(a.err);
        if (e != 0) st = e;
        a.info->iters = iters;
        a.info->refinements = refinements;
        a.info->status = st;
        a.info->reserved = 0;
        a.info->rel_res_l2 = sqrt(tot[0]) / bnorm;
        a.info->rel_res_l1 = l1[0] / (l1[1] + 1e-300);
    }
}

__device__ void record_abort(const SolveArgs &a)
{
    // Reached only when a barrier failed; the CTA that failed has recorded the
    // cause in *err.  CTA 0 writes what it knows.
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.info->status = ld_volatile_i32(a.err);
        a.info->rel_res_l2 = -1.0;
        a.info->rel_res_l1 = -1.0;
    }
}

enum Action : int { kGo = 0, kConverged = 1, kCheck = 2, kNotConverged = 3, kBreakdown = 4, kUpdate = 5, kRestart = 6 };

}  // namespace

// ---------------------------------------------------------------------------
// FP64 Jacobi-PCG
// ---------------------------------------------------------------------------
template <int CH, int TPB>
__global__ void __launch_bounds__(TPB, 1) k_solve_fp64(SolveArgs a)
{
    __shared__ Shared sh;
    Grid g{a.bar, a.err, a.partials, a.budget_ns, 0u, (int)gridDim.x, 0};
    const Range R = my_range(a.m.n_slices);
    const int n = a.m.n;
    double *x = a.x64;  // gathered by the true-residual pass
    double *__restrict__ r = a.r64;
    double *p = a.p64;  // gathered by the SpMV: read by other CTAs, no nc loads
    double *__restrict__ q = a.q64;
    const double *__restrict__ dinv = a.dinv64;
    // thread-0 scalar state
    double bnorm = 1.0, rz = 0.0;
    int checks = 0;

    if (a.use_x0) {
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) x[i] = a.p_user[a.iperm[i]];
        }
        if (!grid_sync(g, sh)) { record_abort(a); return; }
    }
    // r = b - A x, z = D^{-1} r, p = z
    double v3[3] = {0.0, 0.0, 0.0};  // b.b, r.r, r.z
    for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
        const int i = s * kSlice + R.lane;
        if (i < n) {
            const double bi = a.b[i];
            double ri = bi;
            if (a.use_x0) ri = bi - apply64_diag<CH>(a.m, row_of(a.m, s), R.lane, x, x[i], a.diag64[i]);
            else x[i] = 0.0;
            const double zi = dinv[i] * ri;
            r[i] = ri;
            p[i] = zi;
            v3[0] += bi * bi;
            v3[1] += ri * ri;
            v3[2] += ri * zi;
        }
    }
    block_sum_f64<3>(sh, v3);
    double t3[3];
    if (!grid_allreduce<3>(g, sh, v3, t3)) { record_abort(a); return; }
    if (threadIdx.x == 0) {
        bnorm = (t3[0] > 0.0) ? sqrt(t3[0]) : 1.0;
        rz = t3[2];
        sh.ctl.action = (sqrt(t3[1]) / bnorm <= a.rtol) ? kConverged : kGo;
    }
    __syncthreads();
    int action = sh.ctl.action;
    int iters = 0, status = GFM_OK;
    while (action != kConverged) {
        if (iters >= a.max_iters) { status = GFM_ERR_NOT_CONVERGED; break; }
        if (!grid_sync(g, sh)) { record_abort(a); return; }  // p complete
        // pass 1: q = A p, p.q
        double v1[1] = {0.0};
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) {
                const double pi = p[i];
                const double qi = apply64_diag<CH>(a.m, row_of(a.m, s), R.lane, p, pi, a.diag64[i]);
                q[i] = qi;
                v1[0] += pi * qi;
            }
        }
        block_sum_f64<1>(sh, v1);
        double t1[1];
        if (!grid_allreduce<1>(g, sh, v1, t1)) { record_abort(a); return; }
        if (threadIdx.x == 0) {
            const double pq = t1[0];
            const bool ok = pq > 0.0 && isfinite(pq);
            sh.ctl.alpha = ok ? rz / pq : 0.0;
            sh.ctl.action = ok ? kGo : kBreakdown;
        }
        __syncthreads();
        if (sh.ctl.action == kBreakdown) { status = GFM_ERR_BREAKDOWN; break; }
        const double alpha = sh.ctl.alpha;
        // pass 2: x += alpha p, r -= alpha q, z = D^{-1} r; r.z, r.r
        double v2[2] = {0.0, 0.0};
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) {
                x[i] = fma(alpha, p[i], x[i]);
                const double ri = fma(-alpha, q[i], r[i]);
                r[i] = ri;
                const double zi = dinv[i] * ri;
                v2[0] += ri * zi;
                v2[1] += ri * ri;
            }
        }
        block_sum_f64<2>(sh, v2);
        double t2[2];
        if (!grid_allreduce<2>(g, sh, v2, t2)) { record_abort(a); return; }
        ++iters;
        if (threadIdx.x == 0) {
            if (sqrt(t2[1]) / bnorm <= a.rtol) {
                sh.ctl.action = kCheck;
            } else {
                sh.ctl.beta = t2[0] / rz;
                rz = t2[0];
                sh.ctl.action = kGo;
            }
        }
        __syncthreads();
        action = sh.ctl.action;
        if (action == kCheck) {
            // confirm with the true residual; restart from it on a miss
            if (!grid_sync(g, sh)) { record_abort(a); return; }  // x complete
            double vt[2] = {0.0, 0.0};
            for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
                const int i = s * kSlice + R.lane;
                if (i < n) {
                    const double ri = a.b[i] - apply64_diag<CH>(a.m, row_of(a.m, s), R.lane, x, x[i], a.diag64[i]);
                    const double zi = dinv[i] * ri;
                    r[i] = ri;
                    p[i] = zi;
                    vt[0] += ri * zi;
                    vt[1] += ri * ri;
                }
            }
            block_sum_f64<2>(sh, vt);
            double tt[2];
            if (!grid_allreduce<2>(g, sh, vt, tt)) { record_abort(a); return; }
            if (threadIdx.x == 0) {
                ++checks;
                rz = tt[0];
                if (sqrt(tt[1]) / bnorm <= a.rtol) sh.ctl.action = kConverged;
                else sh.ctl.action = (checks > a.max_refine) ? kNotConverged : kGo;
            }
            __syncthreads();
            action = sh.ctl.action;
            if (action == kNotConverged) { status = GFM_ERR_NOT_CONVERGED; break; }
            continue;
        }
        const double beta = sh.ctl.beta;
        // pass 3: p = z + beta p
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) p[i] = fma(beta, p[i], dinv[i] * r[i]);
        }
    }
    if (threadIdx.x == 0) sh.ctl.action = checks;
    __syncthreads();
    finish<CH>(a, g, sh, R, iters, sh.ctl.action, status, bnorm);
}

// ---------------------------------------------------------------------------
// Mixed precision: FP32 PCG with FP64 reliable updates
// ---------------------------------------------------------------------------
namespace {

// Residual replacement.  When `fold`, first x += e / sc in FP64 (e = 0).
// Then r = b - A x in FP64 (difference form), r32 = (float)(r sc),
// u = r32 / D into up.x; with `zero_p` the kept direction up.y is cleared.
// t = (||r||^2 in FP64, r32.u, r32.r32).
template <int CH>
__device__ bool replace_residual(const SolveArgs &a, Grid &g, Shared &sh, const Range &R, float2 *up, double sc,
                                 double isc, bool fold, bool zero_p, double (&t)[3])
{
    const int n = a.m.n;
    const int ref = a.prm->ref;
    const double pin64 = a.prm->pin64;
    double *x = a.x64;
    if (fold) {
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) {
                x[i] = fma((double)a.E[i], isc, x[i]);
                a.E[i] = 0.0f;
            }
        }
        if (!grid_sync(g, sh)) return false;  // x complete
    }
    double vr[1] = {0.0};
    FF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
        const int i = s * kSlice + R.lane;
        if (i < n) {
            const double xi = x[i];
            const double ri = a.b[i] - apply64_diff<CH>(a.m, row_of(a.m, s), R.lane, x, xi, i == ref ? pin64 : 0.0);
            vr[0] = fma(ri, ri, vr[0]);
            const float r32 = (float)(ri * sc);
            const float u = r32 * a.dinv32[i];
            a.R32[i] = r32;
            if (zero_p) up[i] = make_float2(u, 0.0f);
            else up[i].x = u;
            ff_add(acc[0], r32 * u);
            ff_add(acc[1], r32 * r32);
        }
    }
    block_sum_f64<1>(sh, vr);
    double ff2[2];
    block_sum_ff<2>(sh, acc, ff2);
    const double blk[3] = {vr[0], ff2[0], ff2[1]};
    return grid_allreduce<3>(g, sh, blk, t);
}

}  // namespace

template <int CH, int TPB>
__global__ void __launch_bounds__(TPB, 1) k_solve_mixed(SolveArgs a)
{
    __shared__ Shared sh;
    Grid g{a.bar, a.err, a.partials, a.budget_ns, 0u, (int)gridDim.x, 0};
    const Range R = my_range(a.m.n_slices);
    const int n = a.m.n;
    const int ref = a.prm->ref;
    const float pin32 = a.prm->pin32;
    float *__restrict__ E = a.E;
    float *__restrict__ R32 = a.R32;
    float *__restrict__ S32 = a.S32;
    const float *__restrict__ dinv = a.dinv32;

    // prologue: x0, e = 0, no direction yet, ||b||
    double vb[1] = {0.0};
    for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
        const int i = s * kSlice + R.lane;
        if (i < n) {
            a.x64[i] = a.use_x0 ? a.p_user[a.iperm[i]] : 0.0;
            E[i] = 0.0f;
            const double bi = a.b[i];
            vb[0] += bi * bi;
        }
    }
    block_sum_f64<1>(sh, vb);
    double tb[1];
    if (!grid_allreduce<1>(g, sh, vb, tb)) { record_abort(a); return; }
    // thread-0 scalar state
    double bnorm = 1.0, gam = 0.0, gam_prev = 1.0, rho_max = 0.0, best_rel2 = 0.0, rho_stop = 0.0;
    int stall = 0;
    if (threadIdx.x == 0) {
        bnorm = (tb[0] > 0.0) ? sqrt(tb[0]) : 1.0;
        // one power-of-two scale for the whole solve, from ||b||: residual
        // entries start near 1 in FP32 and shrink by at most the tolerance,
        // far above FP32 underflow
        int ex;
        frexp(bnorm / sqrt((double)n), &ex);
        sh.ctl.alpha = ldexp(1.0, -ex);
        sh.ctl.beta = ldexp(1.0, ex);
        rho_stop = (a.rtol * bnorm * sh.ctl.alpha) * (a.rtol * bnorm * sh.ctl.alpha);
    }
    __syncthreads();
    const double sc = sh.ctl.alpha, isc = sh.ctl.beta;

    float2 *cur = a.UP0, *nxt = a.UP1;  // cur holds (u, p_old) for the next pass A
    int iters = 0, updates = 0, status = GFM_OK;
    double t[3];
    if (!replace_residual<CH>(a, g, sh, R, cur, sc, isc, false, true, t)) { record_abort(a); return; }
    ++updates;
    if (threadIdx.x == 0) {
        best_rel2 = t[0] / (bnorm * bnorm);
        gam = t[1];
        rho_max = t[2];
        sh.ctl.be = 0.0f;
        sh.ctl.action = (best_rel2 <= a.rtol * a.rtol) ? kConverged : kGo;
    }
    __syncthreads();
    int action = sh.ctl.action;
    while (action != kConverged) {
        const float be = sh.ctl.be;
        // pass A: p = u + beta p (own and, redundantly, neighbours), s = A p, p.s
        FF accA[1] = {{0.f, 0.f}};
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) {
                const Row rw = row_of(a.m, s);
                const float2 v = cur[i];
                const float pi = fmaf(be, v.y, v.x);
                const float pin_i = (i == ref) ? pin32 : 0.0f;
                float si = pin_i * pi;
                for (int k0 = 0; k0 < rw.w; k0 += CH) {
                    int j[CH];
                    float gm[CH];
                    float2 vj[CH];
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        const bool ok = k0 + c < rw.w;
                        const int slot = rw.base + (k0 + c) * kSlice + R.lane;
                        j[c] = ok ? __ldg(a.m.col + slot) : 0;
                        gm[c] = ok ? __ldg(a.m.val32 + slot) : 0.0f;
                    }
#pragma unroll
                    for (int c = 0; c < CH; ++c) vj[c] = (k0 + c < rw.w) ? cur[j[c]] : v;
#pragma unroll
                    for (int c = 0; c < CH; ++c) si = fmaf(gm[c], pi - fmaf(be, vj[c].y, vj[c].x), si);
                }
                nxt[i].y = pi;
                S32[i] = si;
                ff_add(accA[0], pi * si);
            }
        }
        double blkA[1], tA[1];
        block_sum_ff<1>(sh, accA, blkA);
        if (!grid_allreduce<1>(g, sh, blkA, tA)) { record_abort(a); return; }
        if (threadIdx.x == 0) {
            const double ps = tA[0];
            const bool ok = ps > 0.0 && isfinite(ps) && gam > 0.0;
            sh.ctl.al = ok ? (float)(gam / ps) : 0.0f;
            sh.ctl.action = ok ? kGo : kRestart;
        }
        __syncthreads();
        if (sh.ctl.action == kRestart) {
            // breakdown of the FP32 recurrence: restart from the true residual
            if (!replace_residual<CH>(a, g, sh, R, cur, sc, isc, true, true, t)) { record_abort(a); return; }
            ++updates;
            if (threadIdx.x == 0) {
                const double rel2 = t[0] / (bnorm * bnorm);
                gam = t[1];
                rho_max = t[2];
                sh.ctl.be = 0.0f;
                if (rel2 <= a.rtol * a.rtol) sh.ctl.action = kConverged;
                else sh.ctl.action = (++stall > 3) ? kBreakdown : kGo;
            }
            __syncthreads();
            action = sh.ctl.action;
            if (action == kBreakdown) { status = GFM_ERR_BREAKDOWN; break; }
            continue;
        }
        const float al = sh.ctl.al;
        // pass B: e += alpha p, r -= alpha s, u = D^{-1} r; r.u, r.r
        FF accB[2] = {{0.f, 0.f}, {0.f, 0.f}};
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) {
                const float pi = nxt[i].y;
                E[i] = fmaf(al, pi, E[i]);
                const float ri = fmaf(-al, S32[i], R32[i]);
                R32[i] = ri;
                const float ui = ri * dinv[i];
                nxt[i].x = ui;
                ff_add(accB[0], ri * ui);
                ff_add(accB[1], ri * ri);
            }
        }
        double blkB[2], tB[2];
        block_sum_ff<2>(sh, accB, blkB);
        if (!grid_allreduce<2>(g, sh, blkB, tB)) { record_abort(a); return; }
        ++iters;
        { float2 *tmp = cur; cur = nxt; nxt = tmp; }  // cur = (u_new, p)
        if (threadIdx.x == 0) {
            gam_prev = gam;
            gam = tB[0];
            const double rho = tB[1];
            if (rho > rho_max) rho_max = rho;
            if (iters >= a.max_iters) sh.ctl.action = kNotConverged;
            else if (rho <= 1e-2 * rho_max || rho <= rho_stop || !(gam > 0.0)) sh.ctl.action = kUpdate;
            else {
                sh.ctl.be = (float)(gam / gam_prev);
                sh.ctl.action = kGo;
            }
        }
        __syncthreads();
        action = sh.ctl.action;
        if (action == kUpdate || action == kNotConverged) {
            // fold e into x (FP64) and replace r by the true residual; the
            // direction p is kept
            if (!replace_residual<CH>(a, g, sh, R, cur, sc, isc, true, false, t)) { record_abort(a); return; }
            ++updates;
            if (threadIdx.x == 0) {
                const double rel2 = t[0] / (bnorm * bnorm);
                if (rel2 <= a.rtol * a.rtol) {
                    sh.ctl.action = kConverged;
                } else if (sh.ctl.action != kNotConverged) {
                    if (rel2 < 0.25 * best_rel2) { best_rel2 = rel2; stall = 0; }
                    else ++stall;
                    if (stall > 8 || updates > a.max_refine + 1 + (int)(2.0 * log10(1.0 / a.rtol))) {
                        sh.ctl.action = kNotConverged;
                    } else {
                        gam = t[1];
                        rho_max = t[2];
                        sh.ctl.be = (gam > 0.0 && gam_prev > 0.0) ? (float)(gam / gam_prev) : 0.0f;
                        sh.ctl.action = kGo;
                    }
                }
            }
            __syncthreads();
            action = sh.ctl.action;
            if (action == kNotConverged) { status = GFM_ERR_NOT_CONVERGED; break; }
        }
    }
    finish<CH>(a, g, sh, R, iters, updates, status, bnorm);
}

// Instantiations: faces per row chunk (4 for 2D hex meshes, 8 otherwise) and
// the CTA size bound (512 threads may use up to 128 registers without spills;
// 1024 threads are capped at 64).
const void *solver_kernel(Mode m, int max_width, int threads)
{
    const bool big = threads > 512;
    if (max_width <= 4) {
        if (m == Mode::FP64) return big ? (const void *)k_solve_fp64<4, 1024> : (const void *)k_solve_fp64<4, 512>;
        return big ? (const void *)k_solve_mixed<4, 1024> : (const void *)k_solve_mixed<4, 512>;
    }
    if (m == Mode::FP64) return big ? (const void *)k_solve_fp64<8, 1024> : (const void *)k_solve_fp64<8, 512>;
    return big ? (const void *)k_solve_mixed<8, 1024> : (const void *)k_solve_mixed<8, 512>;
}

int solver_max_threads() { return 1024; }

}  // namespace gfm
