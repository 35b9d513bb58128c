// Coarse space of the two-level preconditioner, rebuilt by every assembly.
//
// With a density ratio of 1000 the ghost-fluid Laplacian (Sec. 3.1) couples
// a region of one phase to the rest only through its interface faces, whose
// coefficients are of the order of the heavy phase's, so the Jacobi-scaled
// operator has a few near-null vectors: roughly constant on each large
// connected region of one phase.  Jacobi-PCG spends thousands of iterations
// on a plateau resolving them.  The preconditioner adds the Galerkin
// correction Z (Z^T A Z)^{-1} Z^T on the span Z of those regions' indicator
// vectors; this file finds the regions and forms E = Z^T A Z.
//
// Regions: union-find over the non-interface faces (same phase on both
// sides), linking the larger root under the smaller, so each region's root
// is its smallest cell index whatever the order of the atomic operations.
// The up-to-kMaxCoarse largest regions of at least min_size cells are kept.
#include "gfm_internal.h"

namespace gfm {

namespace {

__device__ __forceinline__ int cc_find(int *parent, int x)
{
    volatile int *P = parent;
    for (;;) {
        const int p = P[x];
        if (p == x) return x;
        const int gp = P[p];
        if (gp != p) P[x] = gp;  // path splitting: gp is an ancestor of x
        x = p;
    }
}

__device__ __forceinline__ void cc_union(int *parent, int a, int b)
{
    for (;;) {
        a = cc_find(parent, a);
        b = cc_find(parent, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(parent + a, a, b) == a) return;
    }
}

__global__ void k_cc_init(int n, int *parent, int *csize)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    parent[i] = i;
    csize[i] = 0;
}

// Faces with both cells of the same phase (kind 0: both dry, 1: both wet).
__global__ void k_cc_hook(int F, const int32_t *__restrict__ owner, const int32_t *__restrict__ nb,
                          const int8_t *__restrict__ kind, int *parent)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F || kind[f] > 1) return;
    cc_union(parent, owner[f], nb[f]);
}

// Region sizes.  The roots are final here, but parent[] is not rewritten
// with them: a concurrent find's path splitting could overwrite such a write
// with an ancestor that is not the root.  Later kernels find the root again.
__global__ void k_cc_count(int n, int *parent, int *csize)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    atomicAdd(csize + cc_find(parent, i), 1);
}

__global__ void k_cc_candidates(int n, const int *__restrict__ parent, const int *__restrict__ csize, int min_size,
                                int *cand, int *counters)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || parent[i] != i || csize[i] < min_size) return;
    const int k = atomicAdd(counters, 1);
    if (k < kMaxCandidates) cand[k] = i;
}

// One warp: pick the up-to-max_k largest regions (ties: smaller root first).
__global__ void k_cc_select(const int *__restrict__ csize, const int *__restrict__ cand, int *counters, int max_k,
                            int ref, Coarse *co)
{
    const int lane = threadIdx.x;
    const int nc = min(counters[0], kMaxCandidates);
    int K = 0;
    int chosen[kMaxCoarse];
    if (ref >= 0) {
        for (int k = 0; k < max_k && k < kMaxCoarse; ++k) {
            long long best = -1;  // key = size * 2^32 + (2^31 - 1 - root)
            for (int t = lane; t < nc; t += 32) {
                const int c = cand[t];
                bool taken = false;
                for (int q = 0; q < K; ++q) taken |= (chosen[q] == c);
                if (taken) continue;
                const long long key = ((long long)csize[c] << 32) | (long long)(0x7fffffff - c);
                if (key > best) best = key;
            }
            for (int off = 16; off; off >>= 1) {
                const long long o = __shfl_xor_sync(0xffffffffu, best, off);
                if (o > best) best = o;
            }
            if (best < 0) break;
            chosen[K++] = 0x7fffffff - (int)(best & 0xffffffffLL);
        }
    }
    if (lane == 0) {
        co->K = K;
        co->n_cand = counters[0];
        co->n_cross = 0;
        co->ref_comp = -1;
        for (int k = 0; k < kMaxCoarse; ++k) {
            co->roots[k] = k < K ? chosen[k] : -1;
            co->sizes[k] = k < K ? csize[chosen[k]] : 0;
        }
        for (int q = 0; q < kMaxCoarse * kMaxCoarse; ++q) {
            co->E[q] = 0.0;
            co->Einv[q] = 0.0;
        }
        counters[1] = 0;
    }
}

__global__ void k_cc_label(int n, int *parent, const int32_t *__restrict__ perm, const Coarse *__restrict__ co,
                           int8_t *comp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = cc_find(parent, i);
    int id = -1;
    for (int k = 0; k < co->K; ++k)
        if (co->roots[k] == r) id = k;
    comp[perm[i]] = (int8_t)id;
}

// Faces joining different coarse regions, listed in ascending face order
// (count per block, scan of the block counts, ordered write), so the list --
// and every sum over it -- is the same at every assembly.
__device__ __forceinline__ bool cross_face(int f, int F, const int32_t *__restrict__ owner,
                                           const int32_t *__restrict__ nb, const int32_t *__restrict__ perm,
                                           const int8_t *__restrict__ comp, int K, int &o, int &v, int &a, int &b)
{
    if (f >= F || K == 0) return false;
    o = perm[owner[f]];
    v = perm[nb[f]];
    a = comp[o];
    b = comp[v];
    return a != b;
}

__global__ void k_cross_count(int F, const int32_t *__restrict__ owner, const int32_t *__restrict__ nb,
                              const int32_t *__restrict__ perm, const int8_t *__restrict__ comp, const Coarse *co,
                              int *bcount)
{
    int o, v, a, b;
    const bool x = cross_face(blockIdx.x * blockDim.x + threadIdx.x, F, owner, nb, perm, comp, co->K, o, v, a, b);
    const int c = __syncthreads_count(x);
    if (threadIdx.x == 0) bcount[blockIdx.x] = c;
}

// One block of 1024 threads: exclusive scan of the block counts; the total
// goes to counters[1].
__global__ void k_cross_scan(int nblk, const int *__restrict__ bcount, int *boff, int *counters)
{
    __shared__ int warp_tot[32];
    const int per = (nblk + blockDim.x - 1) / blockDim.x;
    const int b0 = min(nblk, (int)threadIdx.x * per), b1 = min(nblk, b0 + per);
    int s = 0;
    for (int q = b0; q < b1; ++q) s += bcount[q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = s;
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? warp_tot[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += y;
        }
        warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    int run = inc - s + (warp > 0 ? warp_tot[warp - 1] : 0);
    for (int q = b0; q < b1; ++q) {
        boff[q] = run;
        run += bcount[q];
    }
    if (threadIdx.x == blockDim.x - 1) counters[1] = run;
}

__global__ void k_cross_write(int F, const int32_t *__restrict__ owner, const int32_t *__restrict__ nb,
                              const int32_t *__restrict__ perm, const int8_t *__restrict__ comp,
                              const double *__restrict__ gamma, const Coarse *co, const int *__restrict__ boff,
                              CrossFace *cross, int max_cross)
{
    __shared__ int wcount[32];
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    int o = 0, v = 0, a = 0, b = 0;
    const bool x = cross_face(f, F, owner, nb, perm, comp, co->K, o, v, a, b);
    const unsigned m = __ballot_sync(0xffffffffu, x);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wcount[warp] = __popc(m);
    __syncthreads();
    if (!x) return;
    int pos = boff[blockIdx.x] + __popc(m & ((1u << lane) - 1u));
    for (int w = 0; w < warp; ++w) pos += wcount[w];
    if (pos >= max_cross) return;
    const double g = gamma[f];
    CrossFace c;
    c.o = o;
    c.v = v;
    c.a = (int8_t)a;
    c.b = (int8_t)b;
    c.g32 = (float)g;
    c.g64 = g;
    cross[pos] = c;
}

// E = Z^T A Z over the cross faces (the pin is added at the end), partial
// sums per block in a fixed order: each thread a fixed stretch of the list,
// then warps, then the block.
constexpr int kEBlocks = kCoarseEParts;
constexpr int kEThreads = 256;

__global__ void k_coarse_E(const CrossFace *__restrict__ cross, const int *__restrict__ counters, int max_cross,
                           const Coarse *co, double *epart)
{
    __shared__ double wsum[kEThreads / 32][kMaxCoarse * kMaxCoarse];
    const int nx = min(counters[1], max_cross);
    const int K = co->K;
    double acc[kMaxCoarse * kMaxCoarse];
    for (int q = 0; q < kMaxCoarse * kMaxCoarse; ++q) acc[q] = 0.0;
    const long long per_blk = ((long long)nx + gridDim.x - 1) / gridDim.x;
    const int c0 = (int)min((long long)nx, per_blk * blockIdx.x);
    const int c1 = (int)min((long long)nx, per_blk * (blockIdx.x + 1));
    const int per_thr = (c1 - c0 + blockDim.x - 1) / blockDim.x;
    const int t0 = min(c1, c0 + (int)threadIdx.x * per_thr), t1 = min(c1, t0 + per_thr);
    for (int t = t0; t < t1 && K > 0; ++t) {
        const CrossFace cf = cross[t];
        const double g = cf.g64;
        if (cf.a >= 0) acc[cf.a * kMaxCoarse + cf.a] += g;
        if (cf.b >= 0) acc[cf.b * kMaxCoarse + cf.b] += g;
        if (cf.a >= 0 && cf.b >= 0) {
            acc[cf.a * kMaxCoarse + cf.b] -= g;
            acc[cf.b * kMaxCoarse + cf.a] -= g;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < kMaxCoarse * kMaxCoarse; ++q) {
        double x = acc[q];
        for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) wsum[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < kMaxCoarse * kMaxCoarse) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += wsum[w][threadIdx.x];
        epart[(size_t)blockIdx.x * kMaxCoarse * kMaxCoarse + threadIdx.x] = x;
    }
}

// E from the block partials (fixed order, one entry per thread), pin term,
// Cholesky inverse (thread 0, K <= 8); K = 0 when anything is off
// (cross-face list overflow, E not positive definite).
__global__ void k_coarse_finish(const int8_t *__restrict__ comp, int ref, const DevParams *__restrict__ prm,
                                Coarse *co, const int *counters, int max_cross, const double *__restrict__ epart)
{
    if (threadIdx.x < kMaxCoarse * kMaxCoarse) {
        double x = 0.0;
        for (int b = 0; b < kEBlocks; ++b) x += epart[(size_t)b * kMaxCoarse * kMaxCoarse + threadIdx.x];
        co->E[threadIdx.x] = x;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int K = co->K;
    const int nx = counters[1];
    if (K > 0 && nx > max_cross) K = 0;
    co->n_cross = nx < max_cross ? nx : max_cross;
    co->ref_comp = (ref >= 0 && K > 0) ? comp[ref] : -1;
    if (co->ref_comp >= 0) co->E[co->ref_comp * kMaxCoarse + co->ref_comp] += prm->pin64;
    double L[kMaxCoarse][kMaxCoarse];
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) L[i][j] = 0.0;
    for (int j = 0; j < K && K > 0; ++j) {
        double d = co->E[j * kMaxCoarse + j];
        for (int q = 0; q < j; ++q) d -= L[j][q] * L[j][q];
        if (!(d > 0.0)) {
            K = 0;
            break;
        }
        d = sqrt(d);
        L[j][j] = d;
        for (int i = j + 1; i < K; ++i) {
            double t = co->E[i * kMaxCoarse + j];
            for (int q = 0; q < j; ++q) t -= L[i][q] * L[j][q];
            L[i][j] = t / d;
        }
    }
    // columns of E^{-1}: solve L L^T x = e_c
    for (int c = 0; c < K; ++c) {
        double y[kMaxCoarse];
        for (int i = 0; i < K; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int q = 0; q < i; ++q) t -= L[i][q] * y[q];
            y[i] = t / L[i][i];
        }
        for (int i = K - 1; i >= 0; --i) {
            double t = y[i];
            for (int q = i + 1; q < K; ++q) t -= L[q][i] * y[q];
            y[i] = t / L[i][i];
        }
        for (int i = 0; i < K; ++i) co->Einv[i * kMaxCoarse + c] = y[i];
    }
    co->K = K;
}

// ---- batched handles: one coarse space per tank --------------------------

// One warp per tank: its up-to-max_k (<= kTankCoarse) largest regions among
// the candidates whose root lies in the tank (ties: smaller root first).
__global__ void k_cc_select_tanks(const int *__restrict__ csize, const int *__restrict__ cand, int *counters,
                                  int max_k, const int32_t *__restrict__ coff, const DevParams *__restrict__ tprm,
                                  Coarse *co, TankCoarse *tco)
{
    const int t = blockIdx.x, lane = threadIdx.x;
    const int nc = min(counters[0], kMaxCandidates);
    const int lo = coff[t], hi = coff[t + 1];
    int K = 0;
    int chosen[kTankCoarse];
    if (tprm[t].ref >= 0) {
        for (int k = 0; k < max_k && k < kTankCoarse; ++k) {
            long long best = -1;  // key = size * 2^32 + (2^31 - 1 - root)
            for (int q = lane; q < nc; q += 32) {
                const int c = cand[q];
                if (c < lo || c >= hi) continue;
                bool taken = false;
                for (int j = 0; j < K; ++j) taken |= (chosen[j] == c);
                if (taken) continue;
                const long long key = ((long long)csize[c] << 32) | (long long)(0x7fffffff - c);
                if (key > best) best = key;
            }
            for (int off = 16; off; off >>= 1) {
                const long long o = __shfl_xor_sync(0xffffffffu, best, off);
                if (o > best) best = o;
            }
            if (best < 0) break;
            chosen[K++] = 0x7fffffff - (int)(best & 0xffffffffLL);
        }
    }
    if (lane == 0) {
        TankCoarse &c = tco[t];
        c.K = K;
        c.ref_comp = -1;
        c.x0 = c.x1 = 0;
        for (int k = 0; k < kTankCoarse; ++k) {
            c.roots[k] = k < K ? chosen[k] : -1;
            c.sizes[k] = k < K ? csize[chosen[k]] : 0;
        }
        for (int q = 0; q < kTankCoarse * kTankCoarse; ++q) c.E[q] = c.Einv[q] = 0.0;
        if (t == 0) {  // the cross-face kernels run when any tank may have regions
            co->K = 1;
            co->n_cand = counters[0];
            co->n_cross = 0;
            co->ref_comp = -1;
            counters[1] = 0;
        }
    }
}

__global__ void k_cc_label_tanks(int n, int T, int *parent, const int32_t *__restrict__ perm,
                                 const int32_t *__restrict__ coff, const TankCoarse *__restrict__ tco, int8_t *comp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = T;  // the tank t with coff[t] <= i < coff[t+1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (coff[mid] <= i) lo = mid;
        else hi = mid;
    }
    const int r = cc_find(parent, i);
    int id = -1;
    for (int k = 0; k < tco[lo].K; ++k)
        if (tco[lo].roots[k] == r) id = k;
    comp[perm[i]] = (int8_t)id;
}

// One warp per tank: its stretch of the cross-face list (face order puts the
// tanks one after another), E = Z^T A Z summed in a fixed order, the pin,
// and the inverse (K <= 2: closed form, K = 0 if not positive definite).
__global__ void k_coarse_tanks(const CrossFace *__restrict__ cross, const int *__restrict__ counters, int max_cross,
                               const int32_t *__restrict__ ioff, int T, const int8_t *__restrict__ comp,
                               const DevParams *__restrict__ tprm, TankCoarse *tco)
{
    const int t = blockIdx.x, lane = threadIdx.x;
    const int nx = min(counters[1], max_cross);
    auto first_of = [&](int tank) {
        if (tank >= T) return nx;
        int lo = 0, hi = nx;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cross[mid].o < ioff[tank]) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    const int x0 = first_of(t), x1 = first_of(t + 1);
    double e00 = 0.0, e01 = 0.0, e11 = 0.0;
    for (int q = x0 + lane; q < x1; q += 32) {
        const CrossFace cf = cross[q];
        const double g = cf.g64;
        if (cf.a == 0 || cf.b == 0) e00 += g;
        if (cf.a == 1 || cf.b == 1) e11 += g;
        if ((cf.a == 0 && cf.b == 1) || (cf.a == 1 && cf.b == 0)) e01 -= g;
    }
    for (int off = 16; off; off >>= 1) {
        e00 += __shfl_xor_sync(0xffffffffu, e00, off);
        e01 += __shfl_xor_sync(0xffffffffu, e01, off);
        e11 += __shfl_xor_sync(0xffffffffu, e11, off);
    }
    if (lane != 0) return;
    TankCoarse &c = tco[t];
    int K = c.K;
    const int ref = tprm[t].ref;
    const int rc = (K > 0 && ref >= 0) ? comp[ref] : -1;
    double E[4] = {e00, e01, e01, e11};
    if (rc >= 0) E[rc * 3] += tprm[t].pin64;  // E[0] or E[3]
    double inv[4] = {0.0, 0.0, 0.0, 0.0};
    if (K == 1) {
        if (E[0] > 0.0) inv[0] = 1.0 / E[0];
        else K = 0;
    } else if (K == 2) {
        const double det = E[0] * E[3] - E[1] * E[2];
        if (E[0] > 0.0 && det > 0.0) {
            inv[0] = E[3] / det;
            inv[1] = -E[1] / det;
            inv[2] = -E[2] / det;
            inv[3] = E[0] / det;
        } else {
            K = 0;
        }
    }
    for (int q = 0; q < 4; ++q) {
        c.E[q] = E[q];
        c.Einv[q] = inv[q];
    }
    c.K = K;
    c.ref_comp = K > 0 ? rc : -1;
    c.x0 = x0;
    c.x1 = x1;
}

inline int blocks_for(long long work, int threads) { return (int)((work + threads - 1) / threads); }

}  // namespace

cudaError_t launch_coarse(const CoarseArgs &a, cudaStream_t s, int *launches)
{
    const int T = 256;
    cudaError_t e = cudaMemsetAsync(a.counters, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_cc_init<<<blocks_for(a.n, T), T, 0, s>>>(a.n, a.parent, a.csize);
    k_cc_hook<<<blocks_for(a.F, T), T, 0, s>>>(a.F, a.owner, a.neighbour, a.kind, a.parent);
    k_cc_count<<<blocks_for(a.n, T), T, 0, s>>>(a.n, a.parent, a.csize);
    k_cc_candidates<<<blocks_for(a.n, T), T, 0, s>>>(a.n, a.parent, a.csize, a.min_size, a.cand, a.counters);
    if (a.T > 0) {
        k_cc_select_tanks<<<a.T, 32, 0, s>>>(a.csize, a.cand, a.counters, a.max_k, a.coff, a.tprm, a.coarse, a.tco);
        k_cc_label_tanks<<<blocks_for(a.n, T), T, 0, s>>>(a.n, a.T, a.parent, a.perm, a.coff, a.tco, a.comp);
    } else {
        k_cc_select<<<1, 32, 0, s>>>(a.csize, a.cand, a.counters, a.max_k, a.ref, a.coarse);
        k_cc_label<<<blocks_for(a.n, T), T, 0, s>>>(a.n, a.parent, a.perm, a.coarse, a.comp);
    }
    const int nblk = blocks_for(a.F, T);
    k_cross_count<<<nblk, T, 0, s>>>(a.F, a.owner, a.neighbour, a.perm, a.comp, a.coarse, a.bcount);
    k_cross_scan<<<1, 1024, 0, s>>>(nblk, a.bcount, a.boff, a.counters);
    k_cross_write<<<nblk, T, 0, s>>>(a.F, a.owner, a.neighbour, a.perm, a.comp, a.gamma, a.coarse, a.boff, a.cross,
                                     a.max_cross);
    if (a.T > 0) {
        k_coarse_tanks<<<a.T, 32, 0, s>>>(a.cross, a.counters, a.max_cross, a.ioff, a.T, a.comp, a.tprm, a.tco);
        if (launches) *launches += 10;
    } else {
        k_coarse_E<<<kEBlocks, kEThreads, 0, s>>>(a.cross, a.counters, a.max_cross, a.coarse, a.epart);
        k_coarse_finish<<<1, kMaxCoarse * kMaxCoarse, 0, s>>>(a.comp, a.ref, a.prm, a.coarse, a.counters,
                                                             a.max_cross, a.epart);
        if (launches) *launches += 11;
    }
    return cudaGetLastError();
}

}  // namespace gfm
