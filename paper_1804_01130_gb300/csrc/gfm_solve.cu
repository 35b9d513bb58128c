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

constexpr int kMaxNR = kMaxReduce;  // the partials buffer is [2][kMaxNR][grid]

// Values decided by thread 0 and broadcast to the CTA.
struct Ctl {
    double alpha, beta, xavg;
    float gam32;  // MIXED: (float) r.u of the last iteration, for alpha
    float al, be;
    int action;
};

struct Shared {
    unsigned long long mbar[kMaxStages];  // completion barriers of the streamed-table stages
    float2 warp_ff[32][kMaxNR];
    double warp_d[32][kMaxNR];
    double out[kMaxNR];
    Ctl ctl;
    double y[kMaxCoarse];    // thread 0: Z^T r (coarse components of the residual)
    double c64[kMaxCoarse];  // coarse correction E^{-1} Z^T r, broadcast
    float c32[kMaxCoarse];
    float cz[kMaxCoarse + 1];  // fused form: 0, then the FP32 coarse correction of each region
    float zb32[kMaxCoarse];  // this CTA's Z^T (A p) in a pass
    double zb64[kMaxCoarse];
    float zbw32[16][kMaxCoarse];  // the same per warp, summed in warp order
    double zbw64[16][kMaxCoarse];
    float zpin32;  // the pinned cell's share, when this CTA holds it
    double zpin64;
    double Einv[kMaxCoarse * kMaxCoarse];  // staged copy of the coarse inverse
    float Einv32[kMaxCoarse * kMaxCoarse];  // the same in FP32 (the FP32 iterations' coarse correction)
    int flag;
    int flag2;  // a reduction's error check, published with its sums
    int ring_fail;  // a streamed-table stage did not arrive within the budget
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

// Thread 0: arrive at the grid barrier and wait for the other CTAs.  Each
// poll reads the counter and the clock (a register, not a memory access);
// the error flag, a second L2 round trip, only every 16th poll.  Returns
// false on a timeout (recorded) or an error seen while waiting.
__device__ __forceinline__ bool grid_arrive_wait(Grid &g)
{
    red_release_add_u32(g.bar, 1u);
    const unsigned target = g.epoch * (unsigned)g.G;
    unsigned long long t0 = 0;
    for (unsigned k = 0;; ++k) {
        const unsigned v = ld_acquire_u32(g.bar);
        if ((int)(v - target) >= 0) break;
        const unsigned long long now = gtime();
        if (k == 0) t0 = now;
        else if (now - t0 > g.budget) {
            atomicCAS(g.err, 0, (int)GFM_ERR_TIMEOUT);
            return false;
        }
        if ((k & 15u) == 15u && ld_volatile_i32(g.err) != 0) return false;
    }
    __threadfence();
    return true;
}

// Grid-wide barrier.  Returns false if the solve must stop (a timeout here or
// an error recorded by any CTA before the barrier completed).
__device__ __forceinline__ bool grid_sync(Grid &g, Shared &sh)
{
    __syncthreads();
    g.epoch += 1u;
    if (threadIdx.x == 0) {
        int fail = grid_arrive_wait(g) ? 0 : 1;
        if (!fail && ld_volatile_i32(g.err) != 0) fail = 1;
        sh.flag = fail;
    }
    __syncthreads();
    return sh.flag == 0;
}

// Deterministic all-reduce of the first `nr` (<= NR) of NR doubles.  `blk`
// must hold this CTA's partial sums in thread 0.  Warp w sums values w,
// w + warps, ... over all CTAs (lane l takes CTAs l, l+32, ...; then a
// butterfly), identically in every CTA.
template <int NR>
__device__ __forceinline__ bool grid_allreduce(Grid &g, Shared &sh, const double (&blk)[NR], double (&out)[NR],
                                               int nr = NR)
{
    static_assert(NR <= kMaxNR, "grid reduction buffer too small");
    int e = 0;
    __syncthreads();
    g.epoch += 1u;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
            if (k < nr) g.partials[((size_t)g.parity * kMaxNR + k) * g.G + blockIdx.x] = blk[k];
        const bool ok = grid_arrive_wait(g);
        // an error raised before the last arrival: read while the sums are
        // read, checked with them
        e = ok ? ld_volatile_i32(g.err) : 1;
        sh.flag = ok ? 0 : 1;
    }
    __syncthreads();
    if (sh.flag != 0) return false;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < nr; k += nw) {
        const double *src = g.partials + ((size_t)g.parity * kMaxNR + k) * g.G;
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
        if (lane == 0) sh.out[k] = acc;
    }
    if (threadIdx.x == 0) sh.flag2 = e;
    g.parity ^= 1;
    __syncthreads();
    if (sh.flag2 != 0) return false;
#pragma unroll
    for (int k = 0; k < NR; ++k) out[k] = (k < nr) ? sh.out[k] : 0.0;
    return true;
}

// Block reduction of per-thread FP64 partials into thread 0 (fixed order).
template <int NR>
__device__ __forceinline__ void block_sum_f64(Shared &sh, double (&v)[NR])
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
__device__ __forceinline__ void block_sum_ff(Shared &sh, FF (&v)[NR], double (&out)[NR])
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

// The same, leaving thread 0 the double-float pair (hi, lo) of each sum.
template <int NR>
__device__ __forceinline__ void block_sum_ff2(Shared &sh, FF (&v)[NR], float2 (&out)[NR])
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
            out[k] = make_float2(r.hi, r.lo);
        }
    }
}

// Deterministic all-reduce of double-float partials (thread 0's blk, one
// (hi, lo) pair per value) across the grid, in double-float arithmetic: the
// FP32 iterations' sums are double-float already, and on GB300 a warp's FP64
// add costs the FP64 pipe as much as a dozen FP32 instructions, so summing
// 152 partials per value in FP64 in up to 13 warps at once queued on that pipe.
// Same order and structure as grid_allreduce; each sum ends as hi + lo in FP64.
template <int NR>
__device__ __forceinline__ bool grid_allreduce_ff(Grid &g, Shared &sh, const float2 (&blk)[NR], double (&out)[NR],
                                                  int nr = NR)
{
    static_assert(NR <= kMaxNR, "grid reduction buffer too small");
    int e = 0;
    __syncthreads();
    g.epoch += 1u;
    float2 *pp = reinterpret_cast<float2 *>(g.partials);  // one 8-byte slot per value and CTA, as for doubles
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
            if (k < nr) pp[((size_t)g.parity * kMaxNR + k) * g.G + blockIdx.x] = blk[k];
        const bool ok = grid_arrive_wait(g);
        e = ok ? ld_volatile_i32(g.err) : 1;
        sh.flag = ok ? 0 : 1;
    }
    __syncthreads();
    if (sh.flag != 0) return false;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < nr; k += nw) {
        const float2 *src = pp + ((size_t)g.parity * kMaxNR + k) * g.G;
        FF v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int b = lane + 32 * q;
            const float2 t = (b < g.G) ? __ldcg(src + b) : make_float2(0.f, 0.f);
            v[q] = FF{t.x, t.y};
        }
        FF acc = ff_merge(ff_merge(ff_merge(v[0], v[1]), ff_merge(v[2], v[3])),
                          ff_merge(ff_merge(v[4], v[5]), ff_merge(v[6], v[7])));
        for (int b = lane + 256; b < g.G; b += 32) {
            const float2 t = __ldcg(src + b);
            acc = ff_merge(acc, FF{t.x, t.y});
        }
        acc = ff_shfl_tree(acc);
        if (lane == 0) sh.out[k] = (double)acc.hi + (double)acc.lo;
    }
    if (threadIdx.x == 0) sh.flag2 = e;
    g.parity ^= 1;
    __syncthreads();
    if (sh.flag2 != 0) return false;
#pragma unroll
    for (int k = 0; k < NR; ++k) out[k] = (k < nr) ? sh.out[k] : 0.0;
    return true;
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

// A CTA's view of its slices' tables: slice (base, width) for every slice of
// the CTA and the first `cap` of its slots (neighbour index + coefficient)
// staged in shared memory at kernel start.  The tables do not change during
// a solve, so every pass then reads them from shared memory instead of L2.
template <typename V>
struct Tab {
    const int2 *meta;    // [s1 - s0] (global slot base, width)
    const int32_t *col;  // [cap]
    const V *val;        // [cap]
    const int32_t *gcol; // global tables for slots past the cache
    const V *gval;
    int s0, base0, end;  // first slice; slot of its first lane; first uncached slot
    bool full;           // every slot of the range is cached

    __device__ __forceinline__ Row row(int s) const
    {
        const int2 m = meta[s - s0];
        return Row{m.x, m.y};
    }
    __device__ __forceinline__ int c(int slot, int) const { return slot < end ? col[slot - base0] : __ldg(gcol + slot); }
    __device__ __forceinline__ V v(int slot) const { return slot < end ? val[slot - base0] : __ldg(gval + slot); }
};

// Stage the CTA's tables; dynamic shared memory holds meta then col then val.
template <typename V>
__device__ Tab<V> stage_tables(const Sell &m, const V *gval, const Range &R, int cache_cap, int meta_slots,
                               unsigned char *dsm)
{
    Tab<V> t;
    int2 *meta = reinterpret_cast<int2 *>(dsm);
    int32_t *col = reinterpret_cast<int32_t *>(dsm + (size_t)meta_slots * sizeof(int2));
    V *val = reinterpret_cast<V *>(dsm + (size_t)meta_slots * sizeof(int2) + (size_t)cache_cap * sizeof(int32_t));
    const int nsl = R.s1 - R.s0;
    for (int k = threadIdx.x; k < nsl; k += blockDim.x) {
        const int b = __ldg(m.slice_ptr + R.s0 + k);
        meta[k] = make_int2(b, (__ldg(m.slice_ptr + R.s0 + k + 1) - b) >> 5);
    }
    const int base0 = (nsl > 0) ? __ldg(m.slice_ptr + R.s0) : 0;
    const int total = (nsl > 0) ? __ldg(m.slice_ptr + R.s1) - base0 : 0;
    const int cap = min(total, cache_cap);
    for (int k = threadIdx.x; k < cap; k += blockDim.x) {
        col[k] = __ldg(m.col + base0 + k);
        val[k] = __ldg(gval + base0 + k);
    }
    __syncthreads();
    t.meta = meta;
    t.col = col;
    t.val = val;
    t.gcol = m.col;
    t.gval = gval;
    t.s0 = R.s0;
    t.base0 = base0;
    t.end = base0 + cap;
    t.full = cap == total;
    return t;
}

// Streamed tables.  When a CTA's slots do not fit in shared memory, the
// mixed operator pass streams them through a ring of shared-memory stages
// filled by 1D bulk async copies (cp.async.bulk, completion counted in
// bytes on one mbarrier per stage).  A stage holds the (neighbour,
// coefficient) slots of `stage_slices` consecutive slices; while the CTA
// works on stage r the copies of stages r+1 .. r+S-1 are in flight, so the
// largest stream of the pass needs no registers to stay in flight.  As soon
// as a pass ends, the first stages of the next pass are requested.  Slot
// ranges start on 128-byte boundaries (slice bases are multiples of 32 slots)
// and their byte counts are multiples of 128, as bulk copies require.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// L2 policy for data a pass reads once: its lines go first when L2 needs
// room, so the vectors that the neighbour gathers reuse stay resident.
__device__ __forceinline__ unsigned long long l2_evict_first()
{
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar,
                                          unsigned long long pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

struct Ring {
    unsigned char *buf;       // n_stages x (col [cap] | val [cap]), or n_stages x ent [cap] (compact)
    unsigned long long *bar;  // [n_stages]
    const int2 *meta;         // the CTA's staged slice (base, width)
    const int32_t *gcol;
    const float *gval;
    const uint32_t *gent;     // compact table (ct), else unused
    const float *dict;        // compact table: the coefficient dictionary, staged after the stages
    int n_stages, stage_slices, cap, nsl, nr, s0, tab_end;
    int ct;                   // 1: the stages hold the compact table (4 bytes per slot)
    unsigned issued;  // stages requested so far (thread 0 only)
    unsigned used;    // stages consumed so far (every thread)
};

// Stage geometry of round r (slices s0 + r*stage_slices ...).
__device__ __forceinline__ int ring_begin(const Ring &g, int r) { return g.meta[r * g.stage_slices].x; }
__device__ __forceinline__ int ring_end(const Ring &g, int r)
{
    const int e = (r + 1) * g.stage_slices;
    return e < g.nsl ? g.meta[e].x : g.tab_end;
}

// Thread 0: request round r into the next stage of the ring.
__device__ __forceinline__ void ring_issue(Ring &g, int r)
{
    const int st = (int)(g.issued % (unsigned)g.n_stages);
    unsigned long long *bar = g.bar + st;
    const int b = ring_begin(g, r);
    const unsigned bytes = (unsigned)(ring_end(g, r) - b) * 4u;
    if (g.ct) {
        uint32_t *ent = reinterpret_cast<uint32_t *>(g.buf + (size_t)st * g.cap * 4);
        mbar_arrive_expect_tx(bar, bytes);
        if (bytes != 0u) bulk_load(ent, g.gent + b, bytes, bar, l2_evict_first());
        ++g.issued;
        return;
    }
    int32_t *col = reinterpret_cast<int32_t *>(g.buf + (size_t)st * g.cap * 8);
    float *val = reinterpret_cast<float *>(col + g.cap);
    mbar_arrive_expect_tx(bar, 2u * bytes);
    if (bytes != 0u) {
        // the tables stream through once per pass: evict-first in L2 (keeping
        // a share of them resident with evict-last instead was slower on the
        // 256x128x128 box: 108.5 ms with none, 112.5 with a quarter, 115.5
        // with half, as those lines crowd out the gathered vectors)
        const unsigned long long pol = l2_evict_first();
        bulk_load(col, g.gcol + b, bytes, bar, pol);
        bulk_load(val, g.gval + b, bytes, bar, pol);
    }
    ++g.issued;
}

// Thread 0: request the first stages of a pass.
__device__ __forceinline__ void ring_prefetch(Ring &g)
{
    const int k = min(g.n_stages, g.nr);
    for (int r = 0; r < k; ++r) ring_issue(g, r);
}

// Wait, bounded by `budget` ns, until stage `g.used` has landed.
__device__ __forceinline__ bool ring_wait(const Ring &g, unsigned long long budget)
{
    unsigned long long *bar = g.bar + (g.used % (unsigned)g.n_stages);
    const unsigned par = (g.used / (unsigned)g.n_stages) & 1u;
    if (mbar_try_wait(bar, par)) return true;
    const unsigned long long t0 = gtime();
    while (!mbar_try_wait(bar, par))
        if (gtime() - t0 > budget) return false;
    return true;
}

// Thread 0, before the CTA returns: wait (bounded) for every stage still in
// flight, so no copy lands in shared memory after the CTA has left.
__device__ __forceinline__ void ring_drain(Ring &g, unsigned long long budget)
{
    for (; g.used < g.issued; ++g.used)
        if (!ring_wait(g, budget)) return;
}

// Table view of the stage holding round r.
struct StageTab {
    const int2 *meta;
    const int32_t *col;
    const float *val;
    int s0, begin;

    __device__ __forceinline__ Row row(int s) const
    {
        const int2 m = meta[s - s0];
        return Row{m.x, m.y};
    }
    __device__ __forceinline__ int c(int slot, int) const { return col[slot - begin]; }
    __device__ __forceinline__ float v(int slot) const { return val[slot - begin]; }
};

__device__ __forceinline__ StageTab ring_stage(const Ring &g, int r)
{
    const int st = (int)(g.used % (unsigned)g.n_stages);
    const int32_t *col = reinterpret_cast<const int32_t *>(g.buf + (size_t)st * g.cap * 8);
    return StageTab{g.meta, col, reinterpret_cast<const float *>(col + g.cap), g.s0, ring_begin(g, r)};
}

// Table view of a compact stage: per slot one word, the neighbour as a
// signed 16-bit offset from the slot's own cell and a 16-bit code of its
// coefficient -- an entry of the dictionary (the few off-interface values
// of each geometric class of faces, staged in shared memory) or, for an
// interface face, kEscape: its coefficient is read from the FP32 table in
// global memory, a load issued beside the neighbour gather.  Half the bytes
// of (index, coefficient) per slot.
struct StageTabCT {
    const int2 *meta;
    const uint32_t *ent;
    const float *dict;
    const float *gval;
    int s0, begin;

    __device__ __forceinline__ Row row(int s) const
    {
        const int2 m = meta[s - s0];
        return Row{m.x, m.y};
    }
    __device__ __forceinline__ int c(int slot, int i) const
    {
        return i + (int)(int16_t)(ent[slot - begin] & 0xFFFFu);
    }
    __device__ __forceinline__ float v(int slot) const
    {
        const uint32_t code = ent[slot - begin] >> 16;
        return code != kEscape ? dict[code] : __ldg(gval + slot);
    }
};

__device__ __forceinline__ StageTabCT ring_stage_ct(const Ring &g, int r)
{
    const int st = (int)(g.used % (unsigned)g.n_stages);
    const uint32_t *ent = reinterpret_cast<const uint32_t *>(g.buf + (size_t)st * g.cap * 4);
    return StageTabCT{g.meta, ent, g.dict, g.gval, g.s0, ring_begin(g, r)};
}

// Set up the ring after stage_tables (the slice metadata is in shared
// memory).  n_stages = 0: tables are read from the static cache / L2.  With
// `ct` the stages hold the compact table and the dictionary is staged after
// them for the whole solve.
__device__ Ring make_ring(const SolveArgs &a, const Range &R, const int2 *meta, unsigned char *dsm, Shared &sh,
                          bool ct = false)
{
    Ring g{};
    g.n_stages = a.n_stages;
    if (g.n_stages <= 0) return g;
    g.buf = dsm + (size_t)a.meta_slots * sizeof(int2);
    g.bar = sh.mbar;
    g.meta = meta;
    g.gcol = a.m.col;
    g.gval = a.m.val32;
    g.gent = a.m.ent;
    g.ct = ct ? 1 : 0;
    if (ct) {
        float *d = reinterpret_cast<float *>(g.buf + (size_t)a.n_stages * a.stage_cap * 4);
        for (int k = threadIdx.x; k < a.m.n_dict; k += blockDim.x) d[k] = __ldg(a.m.dict + k);
        g.dict = d;
    }
    g.stage_slices = a.stage_slices;
    g.cap = a.stage_cap;
    g.s0 = R.s0;
    g.nsl = R.s1 - R.s0;
    g.nr = (g.nsl + g.stage_slices - 1) / g.stage_slices;
    g.tab_end = g.nsl > 0 ? meta[g.nsl - 1].x + kSlice * meta[g.nsl - 1].y : 0;
    if (threadIdx.x == 0) {
        for (int k = 0; k < g.n_stages; ++k) mbar_init(g.bar + k, 1u);
        sh.ring_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    return g;
}

// Point an idle ring (every stage issued has been consumed or drained) at
// the `nsl` slices from s0, whose metadata is staged at `meta`.
__device__ __forceinline__ void ring_retarget(Ring &g, int s0, int nsl, const int2 *meta)
{
    g.meta = meta;
    g.s0 = s0;
    g.nsl = nsl;
    g.nr = (nsl + g.stage_slices - 1) / g.stage_slices;
    g.tab_end = nsl > 0 ? meta[nsl - 1].x + kSlice * meta[nsl - 1].y : 0;
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

// The difference form for UR rows at once (slices s[u], inactive rows give
// pin_i x_i): every row's table and neighbour loads are in flight together,
// so UR rows cost the dependent round trips of one.
template <int CH, int UR>
__device__ __forceinline__ void apply64_diff_multi(const Sell &m, const Row (&rw)[UR], int lane, const double *x,
                                                   const double (&xi)[UR], const double (&pin)[UR],
                                                   double (&acc)[UR])
{
    int wmax = 0;
#pragma unroll
    for (int u = 0; u < UR; ++u) {
        acc[u] = pin[u] * xi[u];
        wmax = max(wmax, rw[u].w);
    }
    for (int k0 = 0; k0 < wmax; k0 += CH) {
        int j[UR][CH];
        double gm[UR][CH], xj[UR][CH];
#pragma unroll
        for (int u = 0; u < UR; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const bool ok = k0 + c < rw[u].w;
                const int slot = rw[u].base + (k0 + c) * kSlice + lane;
                j[u][c] = ok ? __ldg(m.col + slot) : 0;
                gm[u][c] = ok ? __ldg(m.val64 + slot) : 0.0;
            }
#pragma unroll
        for (int u = 0; u < UR; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) xj[u][c] = (k0 + c < rw[u].w) ? x[j[u][c]] : xi[u];
#pragma unroll
        for (int u = 0; u < UR; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) acc[u] = fma(gm[u][c], xi[u] - xj[u][c], acc[u]);
    }
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

// Final two passes shared by both kernels: the true FP64 residual (difference
// form), the solution written in caller order, the OpenFOAM-style normalised
// L1 residual sum|r| / (sum|A x - x_avg rowsum| + sum|b - x_avg rowsum|),
// and the result record.  bnorm is only meaningful in thread 0.
template <int CH>
__device__ __noinline__ void finish(const SolveArgs &a, Grid &g, Shared &sh, const Range &R, int iters, int refinements,
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

// Warp 0, all lanes: c = E^{-1} y (y in shared memory), lane i forming row
// i, published in shared memory in FP64 and FP32.  An FP64 instruction takes
// the same pipe time on GB300 whether one lane or 32 are active, so rows in
// parallel cost K instructions where one thread doing all of them cost K^2.
__device__ __forceinline__ void coarse_solve_warp(int K, Shared &sh)
{
    __syncwarp();
    const int i = threadIdx.x & 31;
    if (i < K) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < kMaxCoarse; ++j)
            if (j < K) t = fma(sh.Einv[i * kMaxCoarse + j], sh.y[j], t);
        sh.c64[i] = t;
        sh.c32[i] = (float)t;
    }
    __syncwarp();
}

// Copy E^{-1} into shared memory once per solve.
__device__ __forceinline__ void stage_coarse(const Coarse *co, Shared &sh)
{
    for (int q = threadIdx.x; q < kMaxCoarse * kMaxCoarse; q += blockDim.x) {
        sh.Einv[q] = co->Einv[q];
        sh.Einv32[q] = (float)co->Einv[q];
    }
}

// One warp, all lanes: lane k < K returns c_k = sum_j E^{-1}_kj y_j in FP32,
// y_j taken from lane j's y (lanes >= K return 0).  The FP32 iterations only
// need the correction in FP32, and on GB300 a chain of K dependent FP64
// multiply-adds costs several times this shuffle-and-FMA form.
__device__ __forceinline__ float coarse32_lane(int K, double y_lane, const Shared &sh)
{
    const int k = threadIdx.x & 31;
    const float yl = (float)y_lane;
    float c = 0.0f;
#pragma unroll
    for (int j = 0; j < kMaxCoarse; ++j) {
        const float yj = __shfl_sync(0xffffffffu, yl, j);
        if (j < K && k < K) c = fmaf(sh.Einv32[k * kMaxCoarse + j], yj, c);
    }
    return c;
}

__device__ __forceinline__ void zero_bins(Shared &sh)
{
    if (threadIdx.x < kMaxCoarse) {
        sh.zb32[threadIdx.x] = 0.0f;
        sh.zb64[threadIdx.x] = 0.0;
    }
    if (threadIdx.x == 0) {
        sh.zpin32 = 0.0f;
        sh.zpin64 = 0.0;
    }
}

// Z^T (A p) over this CTA's share of the faces between coarse regions:
// val(face) = gamma_f (p_own - p_nb) is added to the owner's region and
// subtracted from the neighbour's.  Sums stay in registers per thread (one
// per region), then per warp into wbins[warp], which finish_bins adds in
// warp order: the same result at every run, and no shared-memory atomics
// serialised on the two words of the water/air region pair.
template <typename T, typename ValFn>
__device__ __forceinline__ void cross_sums_range(const CrossFace *cross, int f0, int f1, int K,
                                                 T (*wbins)[kMaxCoarse], ValFn val)
{
    T acc[kMaxCoarse];
#pragma unroll
    for (int k = 0; k < kMaxCoarse; ++k) acc[k] = T(0);
    // taken by the CTA's last threads first, whose warps hold the fewest slices
    const int t0 = f0 + (int)(blockDim.x - 1 - threadIdx.x);
    for (int t = t0; t < f1; t += blockDim.x) {
        const CrossFace cf = cross[t];
        const T v = val(cf);
        if constexpr (sizeof(T) == 4) {
            // FP32: selects are cheaper than a local-memory bin
#pragma unroll
            for (int k = 0; k < kMaxCoarse; ++k) acc[k] += (cf.a == k ? v : T(0)) - (cf.b == k ? v : T(0));
        } else {
            // FP64: two adds into a (local-memory) bin instead of 16 FP64 selects and adds
            if (cf.a >= 0) acc[cf.a] += v;
            if (cf.b >= 0) acc[cf.b] -= v;
        }
    }
    const bool any = __any_sync(0xffffffffu, t0 < f1);  // a warp without faces adds nothing
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kMaxCoarse; ++k) {
        if (k >= K) break;  // K is the same in every thread
        T x = acc[k];
        if (any) {
#pragma unroll
            for (int off = 16; off; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        }
        if (lane == 0) wbins[warp][k] = any ? x : T(0);
    }
}

// The CTA's even share of all n_cross cross faces.
template <typename T, typename ValFn>
__device__ __forceinline__ void cross_sums(const CrossFace *cross, int n_cross, int K, T (*wbins)[kMaxCoarse],
                                           ValFn val)
{
    const int f0 = (int)(((long long)n_cross * blockIdx.x) / gridDim.x);
    const int f1 = (int)(((long long)n_cross * (blockIdx.x + 1)) / gridDim.x);
    cross_sums_range<T>(cross, f0, f1, K, wbins, val);
}

// Warp 0, after a CTA barrier that follows cross_sums: bins[k] = the warps'
// sums in warp order plus the pinned cell's share.
template <typename T>
__device__ __forceinline__ void finish_bins(const T (*wbins)[kMaxCoarse], T pin, int rc, int K, int nw, T *bins)
{
    const int k = threadIdx.x & 31;
    if (k < K) {
        T x = (k == rc) ? pin : T(0);
        for (int w = 0; w < nw; ++w) x += wbins[w][k];
        bins[k] = x;
    }
    __syncwarp();
}

}  // namespace

// ---------------------------------------------------------------------------
// FP64 Jacobi(+coarse)-PCG
// ---------------------------------------------------------------------------
template <int CH>
__global__ void __launch_bounds__(512, 1) k_solve_fp64(SolveArgs a)
{
    // slices per warp in the SpMV pass: one for 4-face rows, two for wider
    // ones (measured best; more unrolled slices only add issue work)
    constexpr int U = CH <= 4 ? 1 : 2;
    __shared__ Shared sh;
    extern __shared__ __align__(16) unsigned char dsm[];
    Grid g{a.bar, a.err, a.partials, a.budget_ns, 0u, (int)gridDim.x, 0};
    const Range R = my_range(a.m.n_slices);
    stage_coarse(a.coarse, sh);
    const Tab<double> tab = stage_tables<double>(a.m, a.m.val64, R, a.cache_cap, a.meta_slots, dsm);
    const int n = a.m.n;
    const int ref = a.prm->ref;
    const int K = a.coarse->K;
    const int rc = a.coarse->ref_comp;
    const double pin64 = a.prm->pin64;
    const int nx = a.coarse->n_cross;
    double *x = a.x64;  // gathered by the true-residual pass
    double *__restrict__ r = a.r64;
    double *p = a.p64;  // gathered by the SpMV: read by other CTAs, no nc loads
    double *__restrict__ q = a.q64;
    const double *__restrict__ dinv = a.dinv64;
    const int8_t *__restrict__ comp = a.comp;
    // thread-0 scalar state (rr_ref: ||r||^2 when Z^T r was last summed exactly;
    // best: smallest true relative residual seen at a check)
    double bnorm = 1.0, rz = 0.0, rr_ref = 0.0, best = 1e300;
    int checks = 0, stall = 0;

    if (a.use_x0) {
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) x[i] = a.p_user[a.iperm[i]];
        }
        if (!grid_sync(g, sh)) { record_abort(a); return; }
    }
    // r = b - A x, p = z = M^{-1} r; with a coarse space the Jacobi part is
    // written first and the coarse part added once Z^T r is known.
    {
        double v3[3] = {0.0, 0.0, 0.0};  // b.b, r.r, r.(D^{-1} r)
        double zb[kMaxCoarse];
#pragma unroll
        for (int k = 0; k < kMaxCoarse; ++k) zb[k] = 0.0;
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
                if (K > 0) {
                    const int cm = comp[i];
#pragma unroll
                    for (int k = 0; k < kMaxCoarse; ++k) zb[k] += (cm == k) ? ri : 0.0;
                }
            }
        }
        block_sum_f64<3>(sh, v3);
        block_sum_f64<kMaxCoarse>(sh, zb);
        double t3[3 + kMaxCoarse];
        {
            double blk[3 + kMaxCoarse];
            blk[0] = v3[0]; blk[1] = v3[1]; blk[2] = v3[2];
            for (int k = 0; k < kMaxCoarse; ++k) blk[3 + k] = zb[k];
            if (!grid_allreduce<3 + kMaxCoarse>(g, sh, blk, t3, 3 + K)) { record_abort(a); return; }
        }
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) {
                bnorm = (t3[0] > 0.0) ? sqrt(t3[0]) : 1.0;
                rz = t3[2];
                rr_ref = t3[1];
                for (int k = 0; k < K; ++k) sh.y[k] = t3[3 + k];
            }
            coarse_solve_warp(K, sh);
            if (threadIdx.x == 0) {
                for (int k = 0; k < K; ++k) rz = fma(sh.c64[k], sh.y[k], rz);
                sh.ctl.action = (sqrt(t3[1]) / bnorm <= a.rtol) ? kConverged : kGo;
            }
        }
        __syncthreads();
        if (K > 0) {
            for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
                const int i = s * kSlice + R.lane;
                if (i < n && comp[i] >= 0) p[i] += sh.c64[comp[i]];
            }
        }
    }
    int action = sh.ctl.action;
    int iters = 0, status = GFM_OK;
    while (action != kConverged) {
        if (iters >= a.max_iters) { status = GFM_ERR_NOT_CONVERGED; break; }
        if (!grid_sync(g, sh)) { record_abort(a); return; }  // p complete
        zero_bins(sh);
        __syncthreads();
        // pass 1: q = A p, p.q; Z^T q from the faces between coarse regions
        double v1[1] = {0.0};
        for (int sb = R.s0 + R.warp; sb < R.s1; sb += U * R.nw) {
            int ii[U], base[U], w[U];
            double pi[U], acc[U];
            int wmax = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int s = sb + u * R.nw;
                ii[u] = s * kSlice + R.lane;
                base[u] = 0;
                w[u] = 0;
                const bool act = s < R.s1 && ii[u] < n;
                if (act) {
                    const Row rw = tab.row(s);
                    base[u] = rw.base;
                    w[u] = rw.w;
                }
                pi[u] = act ? p[ii[u]] : 0.0;
                acc[u] = act ? a.diag64[ii[u]] * pi[u] : 0.0;
                wmax = max(wmax, w[u]);
            }
            for (int k0 = 0; k0 < wmax; k0 += CH) {
                int j[U][CH];
                double gm[U][CH], pj[U][CH];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        const bool ok = k0 + c < w[u];
                        const int slot = base[u] + (k0 + c) * kSlice + R.lane;
                        j[u][c] = ok ? tab.c(slot, 0) : 0;
                        gm[u][c] = ok ? tab.v(slot) : 0.0;
                    }
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int c = 0; c < CH; ++c) pj[u][c] = (k0 + c < w[u]) ? p[j[u][c]] : 0.0;
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int c = 0; c < CH; ++c) acc[u] = fma(-gm[u][c], pj[u][c], acc[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (sb + u * R.nw < R.s1 && ii[u] < n) {
                    q[ii[u]] = acc[u];
                    v1[0] = fma(pi[u], acc[u], v1[0]);
                    if (ii[u] == ref && rc >= 0 && K > 0) sh.zpin64 = pin64 * pi[u];  // pin term of Z^T A p
                }
            }
        }
        if (K > 0)  // each CTA takes an even share of the cross faces
            cross_sums<double>(a.cross, nx, K, sh.zbw64,
                               [&](const CrossFace &cf) { return cf.g64 * (p[cf.o] - p[cf.v]); });
        block_sum_f64<1>(sh, v1);
        if (K > 0 && threadIdx.x < 32) finish_bins<double>(sh.zbw64, sh.zpin64, rc, K, R.nw, sh.zb64);
        double t1[1 + kMaxCoarse];
        {
            double blk[1 + kMaxCoarse];
            blk[0] = v1[0];
            for (int k = 0; k < kMaxCoarse; ++k) blk[1 + k] = sh.zb64[k];
            if (K > 0) {
                if (!grid_allreduce<1 + kMaxCoarse>(g, sh, blk, t1, 1 + K)) { record_abort(a); return; }
            } else {
                double b1[1] = {blk[0]}, o1[1];
                if (!grid_allreduce<1>(g, sh, b1, o1)) { record_abort(a); return; }
                t1[0] = o1[0];
            }
        }
        if (threadIdx.x == 0) {
            const double pq = t1[0];
            const bool ok = pq > 0.0 && isfinite(pq);
            const double alpha = ok ? rz / pq : 0.0;
            sh.ctl.alpha = alpha;
            sh.ctl.action = ok ? kGo : kBreakdown;
            for (int k = 0; k < K; ++k) sh.y[k] = fma(-alpha, t1[1 + k], sh.y[k]);
        }
        __syncthreads();
        if (sh.ctl.action == kBreakdown) { status = GFM_ERR_BREAKDOWN; break; }
        const double alpha = sh.ctl.alpha;
        // pass 2: x += alpha p, r -= alpha q, z = M^{-1} r; r.z, r.r
        double v2[2] = {0.0, 0.0};
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) {
                x[i] = fma(alpha, p[i], x[i]);
                const double ri = fma(-alpha, q[i], r[i]);
                r[i] = ri;
                v2[0] = fma(ri, dinv[i] * ri, v2[0]);  // r.(D^{-1} r); the coarse part is added below
                v2[1] = fma(ri, ri, v2[1]);
            }
        }
        block_sum_f64<2>(sh, v2);
        double t2[2];
        if (!grid_allreduce<2>(g, sh, v2, t2)) { record_abort(a); return; }
        ++iters;
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) {
                if (sqrt(t2[1]) / bnorm <= a.rtol) {
                    sh.ctl.action = kCheck;
                } else if (K > 0 && t2[1] <= 1e-2 * rr_ref) {
                    // the residual fell a decade since Z^T r was last summed:
                    // sum it exactly again so the recurrence cannot drift
                    sh.ctl.xavg = t2[0];
                    rr_ref = t2[1];
                    sh.ctl.action = kUpdate;
                } else {
                    sh.ctl.action = kGo;
                }
            }
            __syncwarp();
            if (sh.ctl.action == kGo) {
                // z = D^{-1} r + Z E^{-1} y:  r.z = r.D^{-1}r + y.E^{-1}y
                coarse_solve_warp(K, sh);
                if (threadIdx.x == 0) {
                    double rzn = t2[0];
                    for (int k = 0; k < K; ++k) rzn = fma(sh.c64[k], sh.y[k], rzn);
                    sh.ctl.beta = rzn / rz;
                    rz = rzn;
                }
            }
        }
        __syncthreads();
        action = sh.ctl.action;
        if (action == kUpdate) {
            double zb[kMaxCoarse];
#pragma unroll
            for (int k = 0; k < kMaxCoarse; ++k) zb[k] = 0.0;
            for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
                const int i = s * kSlice + R.lane;
                if (i < n) {
                    const int cm = comp[i];
                    const double ri = r[i];
#pragma unroll
                    for (int k = 0; k < kMaxCoarse; ++k) zb[k] += (cm == k) ? ri : 0.0;
                }
            }
            block_sum_f64<kMaxCoarse>(sh, zb);
            double ty[kMaxCoarse];
            if (!grid_allreduce<kMaxCoarse>(g, sh, zb, ty, K)) { record_abort(a); return; }
            if (threadIdx.x < 32) {
                if (threadIdx.x == 0)
                    for (int k = 0; k < K; ++k) sh.y[k] = ty[k];
                coarse_solve_warp(K, sh);
                if (threadIdx.x == 0) {
                    double rzn = sh.ctl.xavg;
                    for (int k = 0; k < K; ++k) rzn = fma(sh.c64[k], sh.y[k], rzn);
                    sh.ctl.beta = rzn / rz;
                    rz = rzn;
                    sh.ctl.action = kGo;
                }
            }
            __syncthreads();
            action = sh.ctl.action;
        }
        if (action == kCheck) {
            // confirm with the true residual; restart from it on a miss
            if (!grid_sync(g, sh)) { record_abort(a); return; }  // x complete
            double vt[2] = {0.0, 0.0};
            double zb[kMaxCoarse];
#pragma unroll
            for (int k = 0; k < kMaxCoarse; ++k) zb[k] = 0.0;
            for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
                const int i = s * kSlice + R.lane;
                if (i < n) {
                    // the true residual in difference form (sum_f gamma_f (x_i - x_j)):
                    // accurate to rounding of the differences, not of diag_i x_i
                    const double ri = a.b[i] - apply64_diff<CH>(a.m, row_of(a.m, s), R.lane, x, x[i],
                                                                i == ref ? pin64 : 0.0);
                    const double zi = dinv[i] * ri;
                    r[i] = ri;
                    p[i] = zi;
                    vt[0] += ri * zi;
                    vt[1] += ri * ri;
                    if (K > 0) {
                        const int cm = comp[i];
#pragma unroll
                        for (int k = 0; k < kMaxCoarse; ++k) zb[k] += (cm == k) ? ri : 0.0;
                    }
                }
            }
            block_sum_f64<2>(sh, vt);
            block_sum_f64<kMaxCoarse>(sh, zb);
            double tt[2 + kMaxCoarse];
            {
                double blk[2 + kMaxCoarse];
                blk[0] = vt[0]; blk[1] = vt[1];
                for (int k = 0; k < kMaxCoarse; ++k) blk[2 + k] = zb[k];
                if (!grid_allreduce<2 + kMaxCoarse>(g, sh, blk, tt, 2 + K)) { record_abort(a); return; }
            }
            if (threadIdx.x < 32) {
                if (threadIdx.x == 0) {
                    ++checks;
                    rz = tt[0];
                    rr_ref = tt[1];
                    for (int k = 0; k < K; ++k) sh.y[k] = tt[2 + k];
                }
                coarse_solve_warp(K, sh);
            }
            if (threadIdx.x == 0) {
                for (int k = 0; k < K; ++k) rz = fma(sh.c64[k], sh.y[k], rz);
                const double rel = sqrt(tt[1]) / bnorm;
                if (rel < 0.5 * best) { best = rel; stall = 0; }
                else ++stall;
                if (rel <= a.rtol) sh.ctl.action = kConverged;
                else sh.ctl.action = (checks > a.max_refine || stall >= 3) ? kNotConverged : kGo;
            }
            __syncthreads();
            action = sh.ctl.action;
            if (action == kNotConverged) { status = GFM_ERR_NOT_CONVERGED; break; }
            if (action == kGo && K > 0) {
                for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
                    const int i = s * kSlice + R.lane;
                    if (i < n && comp[i] >= 0) p[i] += sh.c64[comp[i]];
                }
            }
            continue;
        }
        const double beta = sh.ctl.beta;
        // pass 3: p = z + beta p
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n) {
                double zi = dinv[i] * r[i];
                if (K > 0 && comp[i] >= 0) zi += sh.c64[comp[i]];
                p[i] = fma(beta, p[i], zi);
            }
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
// Then r = b - A x in FP64 (difference form), r32 = (float)(r sc) and the
// preconditioned residual u = r32 / D + (Z E^{-1} Z^T r32) into up.x; with
// `zero_p` the kept direction up.y is cleared.  Thread 0 gets
// t = (||r||^2 in FP64, r32.u, r32.r32) and sh.y = Z^T r32.
template <int CH>
__device__ __noinline__ bool replace_residual(const SolveArgs &a, Grid &g, Shared &sh, const Range &R, float2 *up,
                                              double sc, double isc, bool fold, bool zero_p, double (&t)[3],
                                              double &y_lane)
{
    const int n = a.m.n;
    const int ref = a.prm->ref;
    const int K = a.coarse->K;
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
    FF acc[2 + kMaxCoarse];
    for (int k = 0; k < 2 + kMaxCoarse; ++k) acc[k] = FF{0.f, 0.f};
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
            const int cm = a.comp[i];
#pragma unroll
            for (int k = 0; k < kMaxCoarse; ++k) ff_add(acc[2 + k], (cm == k) ? r32 : 0.0f);
        }
    }
    block_sum_f64<1>(sh, vr);
    double ffo[2 + kMaxCoarse];
    block_sum_ff<2 + kMaxCoarse>(sh, acc, ffo);
    double blk[3 + kMaxCoarse], tt[3 + kMaxCoarse];
    blk[0] = vr[0];
    for (int k = 0; k < 2 + kMaxCoarse; ++k) blk[1 + k] = ffo[k];
    if (!grid_allreduce<3 + kMaxCoarse>(g, sh, blk, tt, 3 + K)) return false;
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0)
            for (int k = 0; k < K; ++k) sh.y[k] = tt[3 + k];
        coarse_solve_warp(K, sh);  // c in FP64, for r.u below
        // warp 0's register copy of y, and the FP32 correction the FP32
        // iterations apply (the same form as in every iteration)
        y_lane = (R.lane < K) ? tt[3 + R.lane] : 0.0;
        const float c = coarse32_lane(K, y_lane, sh);
        if (R.lane < K) sh.c32[R.lane] = c;
    }
    if (threadIdx.x == 0) {
        double gam = tt[1];
        for (int k = 0; k < K; ++k) gam = fma(sh.c64[k], sh.y[k], gam);
        t[0] = tt[0];
        t[1] = gam;
        t[2] = tt[2];
        sh.ctl.gam32 = (float)gam;
    }
    __syncthreads();
    if (K > 0) {
        for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
            const int i = s * kSlice + R.lane;
            if (i < n && a.comp[i] >= 0) up[i].x += sh.c32[a.comp[i]];
        }
        if (!grid_sync(g, sh)) return false;  // u complete before it is gathered
    }
    return true;
}

// One group of the mixed operator pass: slices sb, sb + nw, ... (U of them,
// those before s_end): p = u + beta p for the cell and, from the gathered
// (u, p) pairs, for its neighbours; s = A p in difference form; p into P32,
// s into S32, p.s into acc (and the pin's share of Z^T A p).  The tables are
// in shared memory (cached or a streamed stage): neighbour indices and
// coefficients are read where they are used, so only the gathered pairs
// occupy registers and all U x CH gathers of a chunk are in flight at once.
template <int CH, int U, typename TabT>
__device__ __forceinline__ void mixed_op_group(const TabT &tab, int sb, int s_end, const Range &R, int n,
                                               const float2 *cur, float *P32, float *S32, float be, int ref,
                                               float pin32, int rc, int K, Shared &sh, FF &acc)
{
    int ii[U], base[U], w[U];
    float2 v[U];
    float pn[U], si[U];
    int wmax = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int s = sb + u * R.nw;
        ii[u] = s * kSlice + R.lane;
        base[u] = 0;
        w[u] = 0;
        const bool act = s < s_end && ii[u] < n;
        if (act) {
            const Row rw = tab.row(s);
            base[u] = rw.base;
            w[u] = rw.w;
        }
        v[u] = act ? cur[ii[u]] : make_float2(0.f, 0.f);
        wmax = max(wmax, w[u]);
    }
    for (int k0 = 0; k0 < wmax; k0 += CH) {
        float2 vj[U][CH];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const bool ok = k0 + c < w[u];
                vj[u][c] = ok ? cur[tab.c(base[u] + (k0 + c) * kSlice + R.lane, ii[u])] : v[u];
            }
        if (k0 == 0) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                pn[u] = fmaf(be, v[u].y, v[u].x);
                si[u] = (ii[u] == ref) ? pin32 * pn[u] : 0.0f;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const float gm = (k0 + c < w[u]) ? tab.v(base[u] + (k0 + c) * kSlice + R.lane) : 0.0f;
                si[u] = fmaf(gm, pn[u] - fmaf(be, vj[u][c].y, vj[u][c].x), si[u]);
            }
    }
    if (wmax == 0) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            pn[u] = fmaf(be, v[u].y, v[u].x);
            si[u] = (ii[u] == ref) ? pin32 * pn[u] : 0.0f;
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (sb + u * R.nw < s_end && ii[u] < n) {
            __stcs(P32 + ii[u], pn[u]);  // read once, by the update pass
            __stcs(S32 + ii[u], si[u]);
            ff_add(acc, pn[u] * si[u]);
            if (ii[u] == ref && rc >= 0 && K > 0) sh.zpin32 = pin32 * pn[u];  // pin term of Z^T A p
        }
    }
}


// The same group for tables read from global memory (a CTA whose slots do not
// fit in shared memory and are not streamed): every index and coefficient of
// a chunk is loaded first, then every gather, so a chunk costs two dependent
// memory round trips.
template <int CH, int U, typename TabT>
__device__ __forceinline__ void mixed_op_group_hoisted(const TabT &tab, int sb, int s_end, const Range &R, int n,
                                                       const float2 *cur, float *P32, float *S32, float be, int ref,
                                                       float pin32, int rc, int K, Shared &sh, FF &acc)
{
    int ii[U], base[U], w[U];
    float2 v[U];
    float pn[U], si[U];
    int wmax = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int s = sb + u * R.nw;
        ii[u] = s * kSlice + R.lane;
        base[u] = 0;
        w[u] = 0;
        const bool act = s < s_end && ii[u] < n;
        if (act) {
            const Row rw = tab.row(s);
            base[u] = rw.base;
            w[u] = rw.w;
        }
        v[u] = act ? cur[ii[u]] : make_float2(0.f, 0.f);
        pn[u] = fmaf(be, v[u].y, v[u].x);
        si[u] = (ii[u] == ref) ? pin32 * pn[u] : 0.0f;
        wmax = max(wmax, w[u]);
    }
    for (int k0 = 0; k0 < wmax; k0 += CH) {
        int j[U][CH];
        float gm[U][CH];
        float2 vj[U][CH];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const bool ok = k0 + c < w[u];
                const int slot = base[u] + (k0 + c) * kSlice + R.lane;
                j[u][c] = ok ? tab.c(slot, ii[u]) : 0;
                gm[u][c] = ok ? tab.v(slot) : 0.0f;
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) vj[u][c] = (k0 + c < w[u]) ? cur[j[u][c]] : v[u];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) si[u] = fmaf(gm[u][c], pn[u] - fmaf(be, vj[u][c].y, vj[u][c].x), si[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (sb + u * R.nw < s_end && ii[u] < n) {
            __stcs(P32 + ii[u], pn[u]);  // read once, by the update pass
            __stcs(S32 + ii[u], si[u]);
            ff_add(acc, pn[u] * si[u]);
            if (ii[u] == ref && rc >= 0 && K > 0) sh.zpin32 = pin32 * pn[u];  // pin term of Z^T A p
        }
    }
}

}  // namespace

struct T0State {
    double bnorm, gam, gam_prev, rho_max, best_rel2, rho_stop;
    int stall, last_upd;
};

template <int CH, bool STREAM, bool CT = false>
__global__ void __launch_bounds__(512, 1) k_solve_mixed(SolveArgs a)
{
    // slices per warp in one operator group with cached tables: one for
    // 4-face rows (the pass is bound by issue, not by a gather round trip:
    // 18.3 -> 16.4 us per iteration on the 1024x512 tank against four)
    constexpr int U = CH <= 4 ? 1 : 16 / CH;
    constexpr int US = CH <= 6 ? 4 : 2;  // the same with streamed tables
    constexpr int UB = 4;       // slices in flight per warp in the update pass
    __shared__ Shared sh;
    extern __shared__ __align__(16) unsigned char dsm[];
    Grid g{a.bar, a.err, a.partials, a.budget_ns, 0u, (int)gridDim.x, 0};
    const Range R = my_range(a.m.n_slices);
    stage_coarse(a.coarse, sh);
    const Tab<float> tab = stage_tables<float>(a.m, a.m.val32, R, a.cache_cap, a.meta_slots, dsm);
    Ring ring{};
    if constexpr (STREAM) ring = make_ring(a, R, tab.meta, dsm, sh, CT);
    // every early return first lets the stages still in flight land
    auto bail = [&]() {
        if constexpr (STREAM)
            if (threadIdx.x == 0) ring_drain(ring, a.budget_ns);
        record_abort(a);
    };
    const int n = a.m.n;
    const int ref = a.prm->ref;
    const float pin32 = a.prm->pin32;
    const int K = a.coarse->K;
    const int rc = a.coarse->ref_comp;
    const int nx = a.coarse->n_cross;
    float *__restrict__ E = a.E;
    float *__restrict__ R32 = a.R32;
    float *__restrict__ S32 = a.S32;
    float *__restrict__ P32 = a.P32;
    const float *__restrict__ dinv = a.dinv32;
    const int8_t *__restrict__ comp = a.comp;

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
    if (!grid_allreduce<1>(g, sh, vb, tb)) { bail(); return; }
    // thread-0 scalar state (last_upd: iteration of the last residual
    // replacement), kept in shared memory rather than in every thread's
    // registers, which the operator pass needs for its gathers in flight
    __shared__ T0State t0s;
    double &bnorm = t0s.bnorm, &gam = t0s.gam, &gam_prev = t0s.gam_prev, &rho_max = t0s.rho_max,
           &best_rel2 = t0s.best_rel2, &rho_stop = t0s.rho_stop;
    int &stall = t0s.stall, &last_upd = t0s.last_upd;
    if (threadIdx.x == 0) {
        bnorm = 1.0;
        gam = 0.0;
        gam_prev = 1.0;
        rho_max = 0.0;
        best_rel2 = 0.0;
        rho_stop = 0.0;
        stall = 0;
        last_upd = 0;
    }
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
    double y_lane = 0.0;  // warp 0: Z^T r (lane k: component k)
    if (!replace_residual<CH>(a, g, sh, R, cur, sc, isc, false, true, t, y_lane)) { bail(); return; }
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
    if constexpr (STREAM)
        if (threadIdx.x == 0) ring_prefetch(ring);
    while (action != kConverged) {
        const float be = sh.ctl.be;
        zero_bins(sh);
        __syncthreads();
        // pass A: p = u + beta p (own and, redundantly, neighbours), s = A p, p.s
        FF accA[1] = {{0.f, 0.f}};
        if constexpr (STREAM) {
            for (int r = 0; r < ring.nr; ++r) {
                if (ring_wait(ring, a.budget_ns)) {
                    const int sr0 = R.s0 + r * ring.stage_slices;
                    const int sr1 = min(R.s1, sr0 + ring.stage_slices);
                    if constexpr (CT) {
                        const StageTabCT st = ring_stage_ct(ring, r);
                        for (int sb = sr0 + R.warp; sb < sr1; sb += US * R.nw)
                            mixed_op_group<CH, US>(st, sb, sr1, R, n, cur, P32, S32, be, ref, pin32, rc, K, sh,
                                                   accA[0]);
                    } else {
                        const StageTab st = ring_stage(ring, r);
                        for (int sb = sr0 + R.warp; sb < sr1; sb += US * R.nw)
                            mixed_op_group<CH, US>(st, sb, sr1, R, n, cur, P32, S32, be, ref, pin32, rc, K, sh,
                                                   accA[0]);
                    }
                } else {
                    sh.ring_fail = 1;
                }
                ++ring.used;
                __syncthreads();  // stage consumed: it may be refilled
                if (sh.ring_fail) break;
                if (threadIdx.x == 0 && r + ring.n_stages < ring.nr) ring_issue(ring, r + ring.n_stages);
            }
            if (sh.ring_fail) {
                if (threadIdx.x == 0) atomicCAS(a.err, 0, (int)GFM_ERR_TIMEOUT);
                bail();
                return;
            }
            // the next pass's first stages load during the rest of the iteration
            if (threadIdx.x == 0) ring_prefetch(ring);
        } else if (tab.full) {
            // the whole range is cached: a view without the per-slot fallback
            // to global memory, so the group's loads carry no branches
            const StageTab ft{tab.meta, tab.col, tab.val, tab.s0, tab.base0};
            for (int sb = R.s0 + R.warp; sb < R.s1; sb += U * R.nw)
                mixed_op_group<CH, U>(ft, sb, R.s1, R, n, cur, P32, S32, be, ref, pin32, rc, K, sh, accA[0]);
        } else {
            for (int sb = R.s0 + R.warp; sb < R.s1; sb += U * R.nw)
                mixed_op_group<CH, U>(tab, sb, R.s1, R, n, cur, P32, S32, be, ref, pin32, rc, K, sh, accA[0]);
        }
        if (K > 0)  // Z^T (A p) from the faces between coarse regions (the pin's share is added above)
            cross_sums<float>(a.cross, nx, K, sh.zbw32, [&](const CrossFace &cf) {
                const float2 vo = cur[cf.o], vv = cur[cf.v];
                return cf.g32 * (fmaf(be, vo.y, vo.x) - fmaf(be, vv.y, vv.x));
            });
        double tA[1 + kMaxCoarse];
        float2 blkA[1];
        block_sum_ff2<1>(sh, accA, blkA);
        if (K > 0) {
            float2 b9[1 + kMaxCoarse];
            b9[0] = blkA[0];
            if (threadIdx.x < 32) finish_bins<float>(sh.zbw32, sh.zpin32, rc, K, R.nw, sh.zb32);
            for (int k = 0; k < kMaxCoarse; ++k) b9[1 + k] = make_float2(sh.zb32[k], 0.0f);
            if (!grid_allreduce_ff<1 + kMaxCoarse>(g, sh, b9, tA, 1 + K)) { bail(); return; }
        } else {
            double o1[1];
            if (!grid_allreduce_ff<1>(g, sh, blkA, o1)) { bail(); return; }
            tA[0] = o1[0];
        }
        if (threadIdx.x < 32) {
            // warp 0: alpha in FP32 (the vectors use it in FP32), lane k
            // updates y_k (FP64) and the warp forms the FP32 coarse
            // correction; FP64 work stays in this one warp (GB300's FP64 pipe
            // would serialise it across all warps of the SM)
            const float ps32 = (float)tA[0], gam32 = sh.ctl.gam32;
            const bool ok = ps32 > 0.0f && isfinite(ps32) && gam32 > 0.0f;
            const float al0 = ok ? gam32 / ps32 : 0.0f;
            if (threadIdx.x == 0) {
                sh.ctl.al = al0;
                sh.ctl.action = ok ? kGo : kRestart;
            }
            double zk = 0.0;  // this lane's (Z^T A p)_k, picked without indexing the array at run time
#pragma unroll
            for (int k = 0; k < kMaxCoarse; ++k)
                if (k == R.lane) zk = tA[1 + k];
            if (R.lane < K) {
                y_lane = fma(-(double)al0, zk, y_lane);
                sh.y[R.lane] = y_lane;
            }
            const float c = coarse32_lane(K, y_lane, sh);
            if (R.lane < K) sh.c32[R.lane] = c;
        }
        __syncthreads();
        if (sh.ctl.action == kRestart) {
            // breakdown of the FP32 recurrence: restart from the true residual
            if (!replace_residual<CH>(a, g, sh, R, cur, sc, isc, true, true, t, y_lane)) { bail(); return; }
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
        // pass B: e += alpha p, r -= alpha s, u = M^{-1} r; r.u, r.r
        FF accB[2] = {{0.f, 0.f}, {0.f, 0.f}};
        for (int sb = R.s0 + R.warp; sb < R.s1; sb += UB * R.nw) {
            int ii[UB];
            bool act[UB];
            float pi[UB], si[UB], ri[UB], ei[UB], di[UB];
            int cm[UB];
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                ii[u] = (sb + u * R.nw) * kSlice + R.lane;
                act[u] = sb + u * R.nw < R.s1 && ii[u] < n;
                // streamed once per iteration: evict-first (the gathered
                // (u, p) pairs are what L2 should keep)
                pi[u] = act[u] ? __ldcs(P32 + ii[u]) : 0.f;
                si[u] = act[u] ? __ldcs(S32 + ii[u]) : 0.f;
                ri[u] = act[u] ? __ldcs(R32 + ii[u]) : 0.f;
                ei[u] = act[u] ? __ldcs(E + ii[u]) : 0.f;
                di[u] = act[u] ? __ldcs(dinv + ii[u]) : 0.f;
                cm[u] = (act[u] && K > 0) ? (int)comp[ii[u]] : -1;
            }
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                if (act[u]) {
                    __stcs(E + ii[u], fmaf(al, pi[u], ei[u]));
                    const float rn = fmaf(-al, si[u], ri[u]);
                    __stcs(R32 + ii[u], rn);
                    float un = rn * di[u];
                    if (cm[u] >= 0) un += sh.c32[cm[u]];
                    nxt[ii[u]] = make_float2(un, pi[u]);
                    ff_add(accB[0], rn * un);
                    ff_add(accB[1], rn * rn);
                }
            }
        }
        double tB[2];
        float2 blkB[2];
        block_sum_ff2<2>(sh, accB, blkB);
        if (!grid_allreduce_ff<2>(g, sh, blkB, tB)) { bail(); return; }
        ++iters;
        { float2 *tmp = cur; cur = nxt; nxt = tmp; }  // cur = (u_new, p)
        if (threadIdx.x == 0) {
            gam_prev = gam;
            gam = tB[0];
            const double rho = tB[1];
            if (rho > rho_max) rho_max = rho;
            // replacement when the FP32 residual fell a decade, claims
            // convergence, or has not fallen a decade for 1000 iterations
            // (a stagnating FP32 recurrence is then caught by the stall test)
            if (iters >= a.max_iters) sh.ctl.action = kNotConverged;
            else if (rho <= 1e-2 * rho_max || rho <= rho_stop || !(gam > 0.0) || iters - last_upd >= 1000) {
                sh.ctl.action = kUpdate;
                last_upd = iters;
            }
            else {
                sh.ctl.be = (float)gam / (float)gam_prev;
                sh.ctl.action = kGo;
            }
            sh.ctl.gam32 = (float)gam;
        }
        __syncthreads();
        action = sh.ctl.action;
        if (action == kUpdate || action == kNotConverged) {
            // fold e into x (FP64) and replace r by the true residual; the
            // direction p is kept
            if (!replace_residual<CH>(a, g, sh, R, cur, sc, isc, true, false, t, y_lane)) { bail(); return; }
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
                        sh.ctl.gam32 = (float)gam;
                    }
                }
            }
            __syncthreads();
            action = sh.ctl.action;
            if (action == kNotConverged) { status = GFM_ERR_NOT_CONVERGED; break; }
        }
    }
    if constexpr (STREAM)
        if (threadIdx.x == 0) ring_drain(ring, a.budget_ns);
    finish<CH>(a, g, sh, R, iters, updates, status, bnorm);
}

// ---------------------------------------------------------------------------
// Mixed precision, fused form: ONE operator pass and ONE grid all-reduce per
// FP32 iteration.
//
// The two-pass iteration needs two grid-wide all-reduces (p.s, then r.u),
// and on a mesh whose vectors stay in L2 those cost more than the passes.
// Here the update of iteration k is folded into the operator pass of
// iteration k + 1.  Each cell keeps the state (q, t, p, region), with
// q = D^{-1} r the Jacobi part of the preconditioned residual and
// t = D^{-1} s, s = A p.  Given alpha_k, beta_{k+1} and the coarse
// correction c_{k+1} = E^{-1} Z^T r_{k+1}, one pass forms, for the cell and,
// from their gathered state, for its neighbours,
//     q' = q - alpha t,   u' = q' + c[region],   p' = u' + beta p,
// then s' = A p' (difference form), t' = s' / D and e += alpha p.  Its
// partial sums are p'.s' (for alpha), q'.D q' = r'.D^{-1} r' (for r'.u'),
// t'.D q' and t'.D t' (so that r''.D^{-1} r'' after the next step, and with
// it beta, follows from alpha without another all-reduce), r'.r' (the
// stopping and replacement tests) and Z^T A p' (the coarse recurrence).  A
// neighbour's p' is recomputed with the same operations as its owner's, so
// both sides of a face use the same bits.  Residual replacement, restarts
// and the stopping rules are those of the two-pass form.
// ---------------------------------------------------------------------------
namespace {

// p' of a cell from its stored state (q, t, p, region bits).
__device__ __forceinline__ float fused_pnew(float4 v, float al, float be, const Shared &sh)
{
    const float qn = fmaf(-al, v.y, v.x);
    return fmaf(be, v.z, __fadd_rn(qn, sh.cz[__float_as_int(v.w) + 1]));
}

// One group of the fused pass: slices sb, sb + nw, ... (U of them, those
// before s_end); acc gets p'.s', q'.D q', t'.D q', t'.D t', r'.r'.
template <int CH, int U, typename TabT>
__device__ __forceinline__ void fused_group(const TabT &tab, int sb, int s_end, const Range &R, int n,
                                            const float4 *__restrict__ cur, float4 *__restrict__ nxt,
                                            float *__restrict__ E, const float *__restrict__ dinv, float al, float be,
                                            int ref, float pin32, int rc, int K, Shared &sh, FF (&acc)[5])
{
    int ii[U], base[U], w[U];
    float4 v[U];
    float pn[U], si[U], di[U], ei[U];
    int wmax = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int s = sb + u * R.nw;
        ii[u] = s * kSlice + R.lane;
        base[u] = 0;
        w[u] = 0;
        const bool act = s < s_end && ii[u] < n;
        if (act) {
            const Row rw = tab.row(s);
            base[u] = rw.base;
            w[u] = rw.w;
        }
        // the cell's own loads all in flight together, before the gathers
        v[u] = act ? cur[ii[u]] : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
        di[u] = act ? __ldcs(dinv + ii[u]) : 0.0f;
        ei[u] = act ? __ldcs(E + ii[u]) : 0.0f;
        wmax = max(wmax, w[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        pn[u] = fused_pnew(v[u], al, be, sh);
        si[u] = (ii[u] == ref) ? pin32 * pn[u] : 0.0f;
    }
    for (int k0 = 0; k0 < wmax; k0 += CH) {
        float4 vj[U][CH];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const bool ok = k0 + c < w[u];
                vj[u][c] = ok ? cur[tab.c(base[u] + (k0 + c) * kSlice + R.lane, ii[u])] : v[u];
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const float gm = (k0 + c < w[u]) ? tab.v(base[u] + (k0 + c) * kSlice + R.lane) : 0.0f;
                si[u] = fmaf(gm, pn[u] - fused_pnew(vj[u][c], al, be, sh), si[u]);
            }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (sb + u * R.nw < s_end && ii[u] < n) {
            const float qn = fmaf(-al, v[u].y, v[u].x);
            const float tn = si[u] * di[u];
            nxt[ii[u]] = make_float4(qn, tn, pn[u], v[u].w);
            __stcs(E + ii[u], fmaf(al, v[u].z, ei[u]));
            const float rn = qn * __frcp_rn(di[u]);  // r' = D q'
            ff_add(acc[0], pn[u] * si[u]);
            ff_add(acc[1], rn * qn);
            ff_add(acc[2], si[u] * qn);
            ff_add(acc[3], si[u] * tn);
            ff_add(acc[4], rn * rn);
            if (ii[u] == ref && rc >= 0 && K > 0) sh.zpin32 = pin32 * pn[u];  // pin term of Z^T A p'
        }
    }
}

// Residual replacement of the fused form.  When `fold`, first x += e / sc in
// FP64 (e = 0).  Then r = b - A x in FP64, r32 = (float)(r sc) and
// q = r32 / D into the state; with `zero_p` the kept direction p and its t
// are cleared.  Every thread gets t = (||r||^2 in FP64, q.D q, t.D q, r32.r32)
// and lane k of warp 0 the k-th component of Z^T r32.
template <int CH>
__device__ __noinline__ bool replace_fused(const SolveArgs &a, Grid &g, Shared &sh, const Range &R, float4 *qd,
                                           double sc, double isc, bool fold, bool zero_p, double (&t)[4],
                                           double &y_lane)
{
    const int n = a.m.n;
    const int ref = a.prm->ref;
    const int K = a.coarse->K;
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
    FF acc[3 + kMaxCoarse];
    for (int k = 0; k < 3 + kMaxCoarse; ++k) acc[k] = FF{0.f, 0.f};
    for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
        const int i = s * kSlice + R.lane;
        if (i < n) {
            const double xi = x[i];
            const double ri = a.b[i] - apply64_diff<CH>(a.m, row_of(a.m, s), R.lane, x, xi, i == ref ? pin64 : 0.0);
            vr[0] = fma(ri, ri, vr[0]);
            const float r32 = (float)(ri * sc);
            const float q = r32 * a.dinv32[i];
            const int cm = a.comp[i];
            float4 v = zero_p ? make_float4(q, 0.0f, 0.0f, __int_as_float(cm)) : qd[i];
            v.x = q;
            qd[i] = v;
            ff_add(acc[0], r32 * q);
            ff_add(acc[1], v.y * r32);
            ff_add(acc[2], r32 * r32);
#pragma unroll
            for (int k = 0; k < kMaxCoarse; ++k) ff_add(acc[3 + k], (cm == k) ? r32 : 0.0f);
        }
    }
    block_sum_f64<1>(sh, vr);
    double ffo[3 + kMaxCoarse];
    block_sum_ff<3 + kMaxCoarse>(sh, acc, ffo);
    double blk[4 + kMaxCoarse], tt[4 + kMaxCoarse];
    blk[0] = vr[0];
    for (int k = 0; k < 3 + kMaxCoarse; ++k) blk[1 + k] = ffo[k];
    // also the barrier after which the next pass gathers the new q
    if (!grid_allreduce<4 + kMaxCoarse>(g, sh, blk, tt, 4 + K)) return false;
    for (int k = 0; k < 4; ++k) t[k] = tt[k];  // every thread: the all-reduced values
    if (threadIdx.x < 32) {
        double yl = 0.0;  // lane k's component, picked without indexing the array at run time
#pragma unroll
        for (int k = 0; k < kMaxCoarse; ++k)
            if (k == R.lane && k < K) yl = tt[4 + k];
        y_lane = yl;
    }
    return true;
}

// Warp 0, K <= 8: y.c = sum over lanes k < K of y_k c_k in FP32 (lanes >= K
// hold zeros, so three butterfly steps sum lanes 0..7), from lane 0 to all.
__device__ __forceinline__ float coarse_dot8(int K, double y_lane, float c)
{
    float yc = ((threadIdx.x & 31) < K) ? (float)y_lane * c : 0.0f;
    yc += __shfl_xor_sync(0xffffffffu, yc, 4);
    yc += __shfl_xor_sync(0xffffffffu, yc, 2);
    yc += __shfl_xor_sync(0xffffffffu, yc, 1);
    return __shfl_sync(0xffffffffu, yc, 0);
}

// Warp 0: r.u of the state, q.D q plus the coarse part y.c with c = E^{-1} y
// in FP32 (the correction the vectors use).  All lanes return the same value.
__device__ __forceinline__ double fused_gamma(int K, double qdq, double y_lane, const Shared &sh)
{
    static_assert(kMaxCoarse <= 8, "coarse_dot8 sums at most 8 lanes");
    return qdq + (double)coarse_dot8(K, y_lane, coarse32_lane(K, y_lane, sh));
}

// Warp 0: one step of the recurrences from state k (gam = r_k.u_k, ps, qdq,
// tdq, tdt = the all-reduced p.s, q.D q, t.D q, t.D t of state k, zk_lane =
// (Z^T A p_k)_lane): alpha_k = gam / p.s in FP32 (the vectors' precision, as
// in the two-pass form), y_{k+1} = y_k - alpha_k Z^T A p_k (FP64),
// c_{k+1} = E^{-1} y_{k+1} into sh.cz, r_{k+1}.u_{k+1} =
// q.D q - 2 alpha t.D q + alpha^2 t.D t + y_{k+1}.c_{k+1} (FP64, where the
// terms cancel) and beta_{k+1} = r_{k+1}.u_{k+1} / gam into sh.ctl.  With
// `restart`, alpha = beta = 0 (the next direction is the preconditioned
// residual).  A non-positive expanded r.u (rounding at a steep drop) also
// sets beta = 0.  FP64 work is kept to a few instructions: GB300's FP64 pipe
// makes each one cost as much as a long FP32 sequence.
__device__ __forceinline__ void fused_advance(int K, double gam, double ps, double qdq, double tdq, double tdt,
                                              double zk_lane, double &y_lane, bool restart, Shared &sh)
{
    const int lane = threadIdx.x & 31;
    float al = 0.0f, be = 0.0f;
    if (!restart) {
        al = (float)gam / (float)ps;
        if (lane < K) y_lane = fma(-(double)al, zk_lane, y_lane);
    }
    const float c = coarse32_lane(K, y_lane, sh);
    if (!restart) {
        const double ad = (double)al;
        const double gn = fma(ad, fma(ad, tdt, -2.0 * tdq), qdq) + (double)coarse_dot8(K, y_lane, c);
        be = (gn > 0.0 && isfinite(gn)) ? (float)gn / (float)gam : 0.0f;
    }
    if (lane < kMaxCoarse) sh.cz[1 + lane] = (lane < K) ? c : 0.0f;
    if (lane == 0) {
        sh.cz[0] = 0.0f;
        sh.ctl.al = al;
        sh.ctl.be = be;
    }
    __syncwarp();
}

}  // namespace

// Thread-0 scalar state of the fused form, in shared memory.
struct FusedState {
    double bnorm, gam, rho_max, best_rel2, rho_stop;
    double ps, tdt;  // p.s and t.D t of the last pass (kept across a replacement)
    int stall, last_upd;
};

template <int CH, bool STREAM>
__global__ void __launch_bounds__(512, 1) k_solve_fused(SolveArgs a)
{
    // slices per warp in one group: two for 4-face rows (22.9 -> 22.4 ms on
    // the 1024x512 tank against one); with more faces the gathered state (16
    // bytes, twice the two-pass form's pair) keeps fewer slices in flight
    constexpr int U = CH <= 4 ? 2 : 8 / CH;
    constexpr int US = CH <= 6 ? 2 : 1;
    __shared__ Shared sh;
    __shared__ FusedState fs;
    extern __shared__ __align__(16) unsigned char dsm[];
    Grid g{a.bar, a.err, a.partials, a.budget_ns, 0u, (int)gridDim.x, 0};
    const Range R = my_range(a.m.n_slices);
    stage_coarse(a.coarse, sh);
    const Tab<float> tab = stage_tables<float>(a.m, a.m.val32, R, a.cache_cap, a.meta_slots, dsm);
    Ring ring{};
    if constexpr (STREAM) ring = make_ring(a, R, tab.meta, dsm, sh, false);
    auto bail = [&]() {
        if constexpr (STREAM)
            if (threadIdx.x == 0) ring_drain(ring, a.budget_ns);
        record_abort(a);
    };
    const int n = a.m.n;
    const int ref = a.prm->ref;
    const float pin32 = a.prm->pin32;
    const int K = a.coarse->K;
    const int rc = a.coarse->ref_comp;
    const int nx = a.coarse->n_cross;
    float *__restrict__ E = a.E;
    const float *__restrict__ dinv = a.dinv32;

    // prologue: x0, e = 0, ||b||
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
    if (!grid_allreduce<1>(g, sh, vb, tb)) { bail(); return; }
    if (threadIdx.x == 0) {
        fs.bnorm = (tb[0] > 0.0) ? sqrt(tb[0]) : 1.0;
        int ex;  // one power-of-two scale for the whole solve, as in the two-pass form
        frexp(fs.bnorm / sqrt((double)n), &ex);
        sh.ctl.alpha = ldexp(1.0, -ex);
        sh.ctl.beta = ldexp(1.0, ex);
        fs.rho_stop = (a.rtol * fs.bnorm * sh.ctl.alpha) * (a.rtol * fs.bnorm * sh.ctl.alpha);
        fs.gam = 0.0;
        fs.rho_max = 0.0;
        fs.best_rel2 = 0.0;
        fs.ps = 0.0;
        fs.tdt = 0.0;
        fs.stall = 0;
        fs.last_upd = 0;
    }
    __syncthreads();
    const double sc = sh.ctl.alpha, isc = sh.ctl.beta;

    float4 *cur = a.Q0, *nxt = a.Q1;  // cur: the state the next pass reads
    int iters = 0, updates = 0, status = GFM_OK;
    double t[4];
    double y_lane = 0.0;   // warp 0: Z^T r of the current state (lane k: component k)
    double zk_lane = 0.0;  // warp 0: Z^T A p of the current state
    if (!replace_fused<CH>(a, g, sh, R, cur, sc, isc, false, true, t, y_lane)) { bail(); return; }
    ++updates;
    if (threadIdx.x < 32) {
        const double gam = fused_gamma(K, t[1], y_lane, sh);
        if (threadIdx.x == 0) {
            fs.best_rel2 = t[0] / (fs.bnorm * fs.bnorm);
            fs.gam = gam;
            fs.rho_max = t[3];
            sh.ctl.action = (fs.best_rel2 <= a.rtol * a.rtol) ? kConverged : kGo;
        }
        fused_advance(K, gam, 0.0, 0.0, 0.0, 0.0, 0.0, y_lane, true, sh);
        zero_bins(sh);
    }
    __syncthreads();
    int action = sh.ctl.action;
    if constexpr (STREAM)
        if (threadIdx.x == 0) ring_prefetch(ring);
    while (action != kConverged) {
        // al, be, sh.cz and the cleared coarse bins were published by warp 0
        // before the CTA barrier that ended the last scalar step
        const float al = sh.ctl.al, be = sh.ctl.be;
        // the fused pass: the update of the last step and s' = A p' of this one
        FF acc[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] = FF{0.f, 0.f};
        if constexpr (STREAM) {
            for (int r = 0; r < ring.nr; ++r) {
                if (ring_wait(ring, a.budget_ns)) {
                    const int sr0 = R.s0 + r * ring.stage_slices;
                    const int sr1 = min(R.s1, sr0 + ring.stage_slices);
                    const StageTab st = ring_stage(ring, r);
                    for (int sb = sr0 + R.warp; sb < sr1; sb += US * R.nw)
                        fused_group<CH, US>(st, sb, sr1, R, n, cur, nxt, E, dinv, al, be, ref, pin32, rc, K, sh, acc);
                } else {
                    sh.ring_fail = 1;
                }
                ++ring.used;
                __syncthreads();  // stage consumed: it may be refilled
                if (sh.ring_fail) break;
                if (threadIdx.x == 0 && r + ring.n_stages < ring.nr) ring_issue(ring, r + ring.n_stages);
            }
            if (sh.ring_fail) {
                if (threadIdx.x == 0) atomicCAS(a.err, 0, (int)GFM_ERR_TIMEOUT);
                bail();
                return;
            }
            if (threadIdx.x == 0) ring_prefetch(ring);
        } else if (tab.full) {
            const StageTab ft{tab.meta, tab.col, tab.val, tab.s0, tab.base0};
            for (int sb = R.s0 + R.warp; sb < R.s1; sb += U * R.nw)
                fused_group<CH, U>(ft, sb, R.s1, R, n, cur, nxt, E, dinv, al, be, ref, pin32, rc, K, sh, acc);
        } else {
            for (int sb = R.s0 + R.warp; sb < R.s1; sb += U * R.nw)
                fused_group<CH, U>(tab, sb, R.s1, R, n, cur, nxt, E, dinv, al, be, ref, pin32, rc, K, sh, acc);
        }
        if (K > 0)  // Z^T (A p') from the faces between coarse regions (the pin's share is added above)
            cross_sums<float>(a.cross, nx, K, sh.zbw32, [&](const CrossFace &cf) {
                return cf.g32 * (fused_pnew(cur[cf.o], al, be, sh) - fused_pnew(cur[cf.v], al, be, sh));
            });
        double tP[5 + kMaxCoarse];
        {
            float2 blk[5], b[5 + kMaxCoarse];
            block_sum_ff2<5>(sh, acc, blk);
            for (int k = 0; k < 5; ++k) b[k] = blk[k];
            if (K > 0 && threadIdx.x < 32) finish_bins<float>(sh.zbw32, sh.zpin32, rc, K, R.nw, sh.zb32);
            for (int k = 0; k < kMaxCoarse; ++k) b[5 + k] = make_float2((K > 0) ? sh.zb32[k] : 0.0f, 0.0f);
            // also the barrier after which the next pass gathers the new state
            if (!grid_allreduce_ff<5 + kMaxCoarse>(g, sh, b, tP, 5 + K)) { bail(); return; }
        }
        ++iters;
        { float4 *tmp = cur; cur = nxt; nxt = tmp; }
        if (threadIdx.x < 32) {
            zero_bins(sh);  // this pass's bins were read before the all-reduce
            double zl = 0.0;
#pragma unroll
            for (int k = 0; k < kMaxCoarse; ++k)
                if (k == R.lane && k < K) zl = tP[5 + k];
            zk_lane = zl;
            const double gam = fused_gamma(K, tP[1], y_lane, sh);
            if (threadIdx.x == 0) {
                const double ps = tP[0], rho = tP[4];
                fs.gam = gam;
                fs.ps = ps;
                fs.tdt = tP[3];
                if (rho > fs.rho_max) fs.rho_max = rho;
                if (iters >= a.max_iters) {
                    sh.ctl.action = kNotConverged;
                } else if (!(ps > 0.0) || !isfinite(ps) || !(gam > 0.0)) {
                    sh.ctl.action = kRestart;  // breakdown of the FP32 recurrence
                } else if (rho <= 1e-2 * fs.rho_max || rho <= fs.rho_stop || iters - fs.last_upd >= 1000) {
                    // replacement when the FP32 residual fell a decade, claims
                    // convergence, or has not fallen a decade for 1000 iterations
                    sh.ctl.action = kUpdate;
                    fs.last_upd = iters;
                } else {
                    sh.ctl.action = kGo;
                }
            }
            __syncwarp();
            if (sh.ctl.action == kGo)
                fused_advance(K, gam, tP[0], tP[1], tP[2], tP[3], zk_lane, y_lane, false, sh);
        }
        __syncthreads();
        action = sh.ctl.action;
        if (action == kGo) continue;
        // fold e into x (FP64) and replace r by the true residual; the
        // direction is kept, or cleared on a restart
        const bool restart = action == kRestart;
        if (!replace_fused<CH>(a, g, sh, R, cur, sc, isc, true, restart, t, y_lane)) { bail(); return; }
        ++updates;
        if (threadIdx.x < 32) {
            // r.u of the state before the replacement: the recurrences' own
            // value, which the step along the kept direction keeps using
            const double gam_pre = fs.gam;
            __syncwarp();
            if (threadIdx.x == 0) {
                const double rel2 = t[0] / (fs.bnorm * fs.bnorm);
                if (rel2 <= a.rtol * a.rtol) {
                    sh.ctl.action = kConverged;
                } else if (restart) {
                    sh.ctl.action = (++fs.stall > 3) ? kBreakdown : kGo;
                } else if (sh.ctl.action != kNotConverged) {
                    if (rel2 < 0.25 * fs.best_rel2) {
                        fs.best_rel2 = rel2;
                        fs.stall = 0;
                    } else {
                        ++fs.stall;
                    }
                    if (fs.stall > 8 || updates > a.max_refine + 1 + (int)(2.0 * log10(1.0 / a.rtol)))
                        sh.ctl.action = kNotConverged;
                    else
                        sh.ctl.action = kGo;
                }
                if (sh.ctl.action == kGo) fs.rho_max = t[3];
            }
            __syncwarp();
            if (sh.ctl.action == kGo) {
                // Residual replacement keeps the recurrences' step: alpha from
                // the pre-replacement r.u and the kept direction's p.s, and beta
                // against the same r.u, while r.u of the next state is expanded
                // from the replaced residual (its q.D q and t.D q) and the kept
                // t.D t.  Taking alpha from the replaced residual's r.u instead
                // let the FP32 recurrence diverge once the true residual sat at
                // its rounding floor: that r.u is no longer the one the kept
                // direction was built for.  After a restart (direction
                // cleared), or when the kept direction cannot give a step, the
                // next direction is the preconditioned residual (alpha = beta = 0).
                const bool fresh = restart || !(fs.ps > 0.0 && gam_pre > 0.0);
                fused_advance(K, gam_pre, fs.ps, t[1], t[2], fs.tdt, zk_lane, y_lane, fresh, sh);
            }
        }
        __syncthreads();
        action = sh.ctl.action;
        if (action == kBreakdown) { status = GFM_ERR_BREAKDOWN; break; }
        if (action == kNotConverged) { status = GFM_ERR_NOT_CONVERGED; break; }
    }
    if constexpr (STREAM)
        if (threadIdx.x == 0) ring_drain(ring, a.budget_ns);
    finish<CH>(a, g, sh, R, iters, updates, status, fs.bnorm);
}

// ---------------------------------------------------------------------------
// Batched mixed-precision solve: many independent tanks in one persistent
// launch.  Every CTA works on one tank at a time; per-tank scalars live in
// shared memory and every CTA computes ALL tanks' sums and decisions from the
// same partials, so all CTAs agree on the barrier schedule without talking:
// each grid step is one iteration of every tank still iterating, residual
// replacements are served in rounds for the tanks that asked, and when tanks
// finish every CTA re-plans the tank->CTA table over the rest.
// ---------------------------------------------------------------------------
namespace {

// Iterations between rounds of residual replacements while a tank waits for one.
constexpr int kReplaceRound = 32;

struct TankState {
    double bnorm[kMaxTanks], sc[kMaxTanks], isc[kMaxTanks], gam[kMaxTanks], gam_prev[kMaxTanks];
    double rho_max[kMaxTanks], best[kMaxTanks], rho_stop[kMaxTanks], xavg[kMaxTanks];
    double tot[6][kMaxTanks];
    float al[kMaxTanks], be[kMaxTanks];
    // each tank's coarse space: K vectors, region of the pinned cell, stretch
    // [x0, x1) of the cross-face list, E^{-1}; y = Z^T r (FP64 recurrence)
    // and the correction c = E^{-1} y (FP32, added to u)
    int K[kMaxTanks], rc[kMaxTanks], x0[kMaxTanks], x1[kMaxTanks];
    // CTAs of each tank [first, last + 1), re-planned when tanks finish, and
    // each tank's slices [sfirst, sfirst + nslc) and end of its real cells
    int2 tcta[kMaxTanks];
    int sfirst[kMaxTanks], nslc[kMaxTanks], tend[kMaxTanks];
    int n_active;
    // tanks with more than kLaneSum CTAs, whose partials a whole warp sums
    int wide[kMaxTanks];
    int n_wide;
    unsigned ring_used;  // thread 0's count of consumed stages after a drain
    double Einv[kTankCoarse * kTankCoarse][kMaxTanks];
    float Einv32[kTankCoarse * kTankCoarse][kMaxTanks];  // the same in FP32 (the FP32 iterations' correction)
    double y[kTankCoarse][kMaxTanks];
    float c32[kTankCoarse][kMaxTanks];
    int act[kMaxTanks];   // kGo while iterating, else kConverged / kNotConverged / kBreakdown
    int flag[kMaxTanks];  // replacement in this iteration: 0, kUpdate, kRestart, kNotConverged
    // a replacement a tank asked for while it can still iterate (kUpdate):
    // it waits for the next replacement round
    int pend[kMaxTanks];
    int wait[kMaxTanks];      // 1: the tank idles until the next replacement round
    int last_rep[kMaxTanks];  // iteration of the tank's last residual replacement
    int iters[kMaxTanks], updates[kMaxTanks], stall[kMaxTanks], last_upd[kMaxTanks], restarts[kMaxTanks];
    int any_flag, any_active;
    int round_age;  // iterations since the last replacement round
};

// Per-tank all-reduce.  Every CTA writes its partials; after the grid
// barrier value k of tank t is the sum over the tank's CTAs in CTA order, by
// one thread when the tank has at most kLaneSum CTAs (its loads all in
// flight at once), else by one warp (lane l takes CTAs l, l + 32, ..., then
// a fixed butterfly), reading the partials straight from L2.  Which rule a tank gets
// depends only on the CTA table, which every CTA holds, so every CTA gets the
// same bits.
template <int NR>
__device__ __forceinline__ bool batch_allreduce(Grid &g, Shared &sh, TankState &ts, const BatchArgs &bt,
                                                const double (&blk)[NR])
{
    static_assert(NR <= kBatchNR && kBatchNR <= kMaxNR, "more values than a batched all-reduce carries");
    int e = 0;
    __syncthreads();
    g.epoch += 1u;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) g.partials[((size_t)g.parity * kMaxNR + k) * g.G + blockIdx.x] = blk[k];
        const bool ok = grid_arrive_wait(g);
        e = ok ? ld_volatile_i32(g.err) : 1;  // checked with the sums, as in grid_allreduce
        sh.flag = ok ? 0 : 1;
    }
    __syncthreads();
    if (sh.flag != 0) return false;
    const int G = g.G, T = bt.T;
    const double *src = g.partials + (size_t)g.parity * kMaxNR * G;
    for (int i = threadIdx.x; i < NR * T; i += blockDim.x) {
        const int k = i / T, t = i - k * T;
        const int2 r = ts.tcta[t];
        const int nc = r.y - r.x;
        if (nc > kLaneSum) continue;
        double v[kLaneSum];
#pragma unroll
        for (int q = 0; q < kLaneSum; ++q) v[q] = (q < nc) ? __ldcg(src + k * G + r.x + q) : 0.0;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < kLaneSum; ++q)
            if (q < nc) acc += v[q];
        ts.tot[k][t] = acc;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < NR * ts.n_wide; i += nw) {
        const int k = i / ts.n_wide, t = ts.wide[i - k * ts.n_wide];
        const int2 r = ts.tcta[t];
        double acc = 0.0;
        for (int c = r.x + lane; c < r.y; c += 32) acc += __ldcg(src + k * G + c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) ts.tot[k][t] = acc;
    }
    if (threadIdx.x == 0) sh.flag2 = e;
    g.parity ^= 1;
    __syncthreads();
    return sh.flag2 == 0;
}

// The same per-tank all-reduce for double-float partials (thread 0's blk,
// one (hi, lo) pair per value), summed per tank in double-float with FP32
// instructions in the same order, each sum converted to FP64 at the end:
// the batched FP32 iterations' sums, which FP64 adds would queue on GB300's
// small FP64 pipe.
template <int NR>
__device__ __forceinline__ bool batch_allreduce_ff(Grid &g, Shared &sh, TankState &ts, const BatchArgs &bt,
                                                   const float2 (&blk)[NR])
{
    static_assert(NR <= kBatchNR && kBatchNR <= kMaxNR, "more values than a batched all-reduce carries");
    int e = 0;
    __syncthreads();
    g.epoch += 1u;
    float2 *pp = reinterpret_cast<float2 *>(g.partials);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) pp[((size_t)g.parity * kMaxNR + k) * g.G + blockIdx.x] = blk[k];
        const bool ok = grid_arrive_wait(g);
        e = ok ? ld_volatile_i32(g.err) : 1;
        sh.flag = ok ? 0 : 1;
    }
    __syncthreads();
    if (sh.flag != 0) return false;
    const int G = g.G, T = bt.T;
    const float2 *src = pp + (size_t)g.parity * kMaxNR * G;
    for (int i = threadIdx.x; i < NR * T; i += blockDim.x) {
        const int k = i / T, t = i - k * T;
        const int2 r = ts.tcta[t];
        const int nc = r.y - r.x;
        if (nc > kLaneSum) continue;
        float2 v[kLaneSum];
#pragma unroll
        for (int q = 0; q < kLaneSum; ++q) v[q] = (q < nc) ? __ldcg(src + k * G + r.x + q) : make_float2(0.f, 0.f);
        FF acc{0.f, 0.f};
#pragma unroll
        for (int q = 0; q < kLaneSum; ++q)
            if (q < nc) acc = ff_merge(acc, FF{v[q].x, v[q].y});
        ts.tot[k][t] = (double)acc.hi + (double)acc.lo;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < NR * ts.n_wide; i += nw) {
        const int k = i / ts.n_wide, t = ts.wide[i - k * ts.n_wide];
        const int2 r = ts.tcta[t];
        FF acc{0.f, 0.f};
        for (int c = r.x + lane; c < r.y; c += 32) {
            const float2 v = __ldcg(src + k * G + c);
            acc = ff_merge(acc, FF{v.x, v.y});
        }
        acc = ff_shfl_tree(acc);
        if (lane == 0) ts.tot[k][t] = (double)acc.hi + (double)acc.lo;
    }
    if (threadIdx.x == 0) sh.flag2 = e;
    g.parity ^= 1;
    __syncthreads();
    return sh.flag2 == 0;
}

// Thread 0: list the tanks whose CTA count calls for a warp-wide sum.
__device__ __forceinline__ void list_wide(TankState &ts, int T)
{
    int n = 0;
    for (int t = 0; t < T; ++t)
        if (ts.tcta[t].y - ts.tcta[t].x > kLaneSum) ts.wide[n++] = t;
    ts.n_wide = n;
}

// One lane, one tank: c = E^{-1} y into ts.c32 (K <= 2); returns y.c.
// The FP32 iterations' form: c = E^{-1} y from the FP32 inverse and the
// rounded y (the vectors apply c in FP32; a chain of FP64 multiply-adds per
// tank costs far more on GB300's FP64 pipe).
__device__ __forceinline__ void tank_coarse_solve32(TankState &ts, int t)
{
    const int K = ts.K[t];
    float yf[kTankCoarse];
#pragma unroll
    for (int j = 0; j < kTankCoarse; ++j) yf[j] = (j < K) ? (float)ts.y[j][t] : 0.0f;
#pragma unroll
    for (int i = 0; i < kTankCoarse; ++i) {
        if (i >= K) break;
        float c = 0.0f;
#pragma unroll
        for (int j = 0; j < kTankCoarse; ++j)
            if (j < K) c = fmaf(ts.Einv32[i * kTankCoarse + j][t], yf[j], c);
        ts.c32[i][t] = c;
    }
}

__device__ __forceinline__ double tank_coarse_solve(TankState &ts, int t)
{
    const int K = ts.K[t];
    double yc = 0.0;
    for (int i = 0; i < K; ++i) {
        double c = 0.0;
        for (int j = 0; j < K; ++j) c = fma(ts.Einv[i * kTankCoarse + j][t], ts.y[j][t], c);
        ts.c32[i][t] = (float)c;
        yc = fma(c, ts.y[i][t], yc);
    }
    return yc;
}

// Residual replacement for the tanks with a pending flag (or all, `all`):
// x += e / sc (FP64, when `fold`), r = b - A x (FP64, difference form),
// r32 = (float)(r sc), u = r32 / D into up (direction cleared on restart).
// ts.tot = (||r||^2, r32.u, r32.r32) per tank.
template <int CH>
__device__ bool batch_replace(const SolveArgs &a, const BatchArgs &bt, Grid &g, Shared &sh, TankState &ts,
                              const Range &R, int tank, int cend, int ref, double pin64, float2 *up, bool fold,
                              bool all)
{
    const bool work = all || ts.flag[tank] != 0;
    const bool zero_p = all || ts.flag[tank] == kRestart;
    const double sc = ts.sc[tank], isc = ts.isc[tank];
    double *x = a.x64;
    if (fold) {
        if (work) {
            // four slices per warp at a time, their loads in flight together
            constexpr int UF = 4;
            for (int sb = R.s0 + R.warp; sb < R.s1; sb += UF * R.nw) {
                float e[UF];
                double xv[UF];
#pragma unroll
                for (int u = 0; u < UF; ++u) {
                    const int i = (sb + u * R.nw) * kSlice + R.lane;
                    const bool act = sb + u * R.nw < R.s1 && i < cend;
                    e[u] = act ? a.E[i] : 0.0f;
                    xv[u] = act ? x[i] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < UF; ++u) {
                    const int i = (sb + u * R.nw) * kSlice + R.lane;
                    if (sb + u * R.nw < R.s1 && i < cend) {
                        x[i] = fma((double)e[u], isc, xv[u]);
                        a.E[i] = 0.0f;
                    }
                }
            }
        }
        if (!grid_sync(g, sh)) return false;  // x complete
    }
    double vr[1] = {0.0};
    FF acc[2 + kTankCoarse] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (work) {
        // two slices per warp at a time: the residual pass is a chain of
        // dependent loads per row (slice table, slots, neighbours)
        constexpr int UR = 2;
        for (int sb = R.s0 + R.warp; sb < R.s1; sb += UR * R.nw) {
            int ii[UR], cm[UR];
            bool act[UR];
            Row rw[UR];
            double xi[UR], bi[UR], pin[UR], ax[UR];
            float di[UR];
#pragma unroll
            for (int u = 0; u < UR; ++u) {
                const int s = sb + u * R.nw;
                ii[u] = s * kSlice + R.lane;
                act[u] = s < R.s1 && ii[u] < cend;
                rw[u] = act[u] ? row_of(a.m, s) : Row{0, 0};
                xi[u] = act[u] ? x[ii[u]] : 0.0;
                bi[u] = act[u] ? a.b[ii[u]] : 0.0;
                di[u] = act[u] ? a.dinv32[ii[u]] : 0.0f;
                cm[u] = act[u] ? (int)a.comp[ii[u]] : -1;
                pin[u] = (act[u] && ii[u] == ref) ? pin64 : 0.0;
            }
            apply64_diff_multi<CH, UR>(a.m, rw, R.lane, x, xi, pin, ax);
#pragma unroll
            for (int u = 0; u < UR; ++u) {
                if (!act[u]) continue;
                const int i = ii[u];
                const double ri = bi[u] - ax[u];
                vr[0] = fma(ri, ri, vr[0]);
                const float r32 = (float)(ri * sc);
                const float uu = r32 * di[u];
                a.R32[i] = r32;
                if (zero_p) up[i] = make_float2(uu, 0.0f);
                else up[i].x = uu;
                ff_add(acc[0], r32 * uu);
                ff_add(acc[1], r32 * r32);
#pragma unroll
                for (int k = 0; k < kTankCoarse; ++k) ff_add(acc[2 + k], (cm[u] == k) ? r32 : 0.0f);
            }
        }
    }
    block_sum_f64<1>(sh, vr);
    double ffo[2 + kTankCoarse];
    block_sum_ff<2 + kTankCoarse>(sh, acc, ffo);
    const double blk[3 + kTankCoarse] = {vr[0], ffo[0], ffo[1], ffo[2], ffo[3]};
    if (!batch_allreduce<3 + kTankCoarse>(g, sh, ts, bt, blk)) return false;
    // replaced tanks: y = Z^T r exactly, c = E^{-1} y, r.z gains y.c, and the
    // coarse correction joins u
    int any_coarse = 0;
    if (threadIdx.x < 32) {
        for (int t = threadIdx.x; t < bt.T; t += 32) {
            if (!(all || ts.flag[t] != 0) || ts.K[t] == 0) continue;
            for (int k = 0; k < ts.K[t]; ++k) ts.y[k][t] = ts.tot[3 + k][t];
            ts.tot[1][t] += tank_coarse_solve(ts, t);
            any_coarse = 1;
        }
        any_coarse = __any_sync(0xffffffffu, any_coarse);
        if (threadIdx.x == 0) sh.flag = any_coarse;
    }
    __syncthreads();
    if (sh.flag == 0) return true;  // the same in every CTA
    __syncthreads();
    if (work && ts.K[tank] > 0) {
        constexpr int UF = 4;  // four slices per warp at a time, their loads in flight together
        for (int sb = R.s0 + R.warp; sb < R.s1; sb += UF * R.nw) {
            int cm[UF];
            float ux[UF];
#pragma unroll
            for (int u = 0; u < UF; ++u) {
                const int i = (sb + u * R.nw) * kSlice + R.lane;
                const bool act = sb + u * R.nw < R.s1 && i < cend;
                cm[u] = act ? (int)a.comp[i] : -1;
                ux[u] = act ? up[i].x : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < UF; ++u) {
                const int i = (sb + u * R.nw) * kSlice + R.lane;
                if (cm[u] >= 0) up[i].x = ux[u] + ts.c32[cm[u]][tank];
            }
        }
    }
    return grid_sync(g, sh);  // u complete before it is gathered
}

// Warp 0 of every CTA: split the grid among the tanks that take part (those
// still iterating, or all of them with `all`).  Each gets one CTA, then the
// CTAs go one at a time to the tank whose CTAs hold the most slices each
// (ties to the lower tank), which minimises the most slices any CTA holds:
// every tank iterates once per grid step, so the step lasts as long as the
// busiest CTA.  Lane l keeps tanks l, l + 32, ...; each step is a warp
// argmax.  A pure function of state every CTA holds, so every CTA builds the
// same table.
__device__ void batch_rebalance(TankState &ts, int T, int G, bool all)
{
    constexpr int PT = kMaxTanks / 32;  // tanks per lane
    const int lane = threadIdx.x & 31;
    int g[PT];
    long long sl[PT];
    int nact = 0;
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int t = lane + 32 * j;
        const bool on = t < T && (all || ts.act[t] == kGo);
        g[j] = on ? 1 : 0;
        sl[j] = on ? ts.nslc[t] : 0;
        nact += on ? 1 : 0;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) nact += __shfl_xor_sync(0xffffffffu, nact, off);
    if (nact == 0) return;
    for (int left = G - nact; left > 0; --left) {
        // this lane's busiest tank (slices per CTA as the fraction bn / bd)
        long long bn = -1;
        int bd = 1, bt = 0x7fffffff;
#pragma unroll
        for (int j = 0; j < PT; ++j)
            if (g[j] > 0 && sl[j] * bd > bn * g[j]) {
                bn = sl[j];
                bd = g[j];
                bt = lane + 32 * j;
            }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const long long on = __shfl_xor_sync(0xffffffffu, bn, off);
            const int od = __shfl_xor_sync(0xffffffffu, bd, off);
            const int ot = __shfl_xor_sync(0xffffffffu, bt, off);
            const long long a = on * bd, b = bn * od;
            if (a > b || (a == b && ot < bt)) {
                bn = on;
                bd = od;
                bt = ot;
            }
        }
        if ((bt & 31) == lane) {
#pragma unroll
            for (int j = 0; j < PT; ++j)
                if (j == (bt >> 5)) g[j] += 1;
        }
    }
#pragma unroll
    for (int j = 0; j < PT; ++j) {
        const int t = lane + 32 * j;
        if (t < T) ts.tcta[t] = make_int2(0, g[j]);  // .y holds the count for now
    }
    __syncwarp();
    if (lane == 0) {
        int c = 0;
        for (int t = 0; t < T; ++t) {
            const int n = ts.tcta[t].y;
            ts.tcta[t] = make_int2(c, c + n);
            c += n;
        }
        list_wide(ts, T);
    }
    __syncwarp();
}

// Slice tables of the batched solve, staged in shared memory like the
// single-mesh ones (the slices' (base, width) and the first slots of the
// range) and staged again whenever a re-plan hands the CTA other slices.  A
// range longer than the metadata area reads the rest of its metadata from
// global memory.
struct BTab {
    const int2 *meta;
    const int32_t *col;
    const float *val;
    const int32_t *gptr, *gcol;
    const float *gval;
    int s0, nmeta, base0, end;
    __device__ __forceinline__ Row row(int s) const
    {
        const int k = s - s0;
        if (k < nmeta) {
            const int2 m = meta[k];
            return Row{m.x, m.y};
        }
        const int b = __ldg(gptr + s);
        return Row{b, (__ldg(gptr + s + 1) - b) >> 5};
    }
    __device__ __forceinline__ int c(int slot, int) const { return slot < end ? col[slot - base0] : __ldg(gcol + slot); }
    __device__ __forceinline__ float v(int slot) const { return slot < end ? val[slot - base0] : __ldg(gval + slot); }
};

// All threads: stage the range's tables (ends with a block barrier; the
// caller makes sure nobody still reads the previous ones).
__device__ BTab stage_btab(const Sell &m, const Range &R, int cache_cap, int meta_slots, unsigned char *dsm)
{
    BTab t;
    int2 *meta = reinterpret_cast<int2 *>(dsm);
    int32_t *col = reinterpret_cast<int32_t *>(dsm + (size_t)meta_slots * sizeof(int2));
    float *val = reinterpret_cast<float *>(dsm + (size_t)meta_slots * sizeof(int2) + (size_t)cache_cap * sizeof(int32_t));
    const int nsl = R.s1 - R.s0;
    const int nmeta = min(nsl, meta_slots);
    for (int k = threadIdx.x; k < nmeta; k += blockDim.x) {
        const int b = __ldg(m.slice_ptr + R.s0 + k);
        meta[k] = make_int2(b, (__ldg(m.slice_ptr + R.s0 + k + 1) - b) >> 5);
    }
    const int base0 = (nsl > 0) ? __ldg(m.slice_ptr + R.s0) : 0;
    const int total = (nsl > 0) ? __ldg(m.slice_ptr + R.s1) - base0 : 0;
    const int cap = min(total, cache_cap);
    for (int k = threadIdx.x; k < cap; k += blockDim.x) {
        col[k] = __ldg(m.col + base0 + k);
        val[k] = __ldg(m.val32 + base0 + k);
    }
    __syncthreads();
    t.meta = meta;
    t.col = col;
    t.val = val;
    t.gptr = m.slice_ptr;
    t.gcol = m.col;
    t.gval = m.val32;
    t.s0 = R.s0;
    t.nmeta = nmeta;
    t.base0 = base0;
    t.end = base0 + cap;
    return t;
}

__device__ void batch_abort(const SolveArgs &a, const BatchArgs &bt)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int e = ld_volatile_i32(a.err);
        for (int t = 0; t < bt.T; ++t) {
            bt.infos[t].status = e;
            bt.infos[t].rel_res_l2 = -1.0;
            bt.infos[t].rel_res_l1 = -1.0;
        }
    }
}

}  // namespace

template <int CH, bool STREAM, bool CT = false>
__global__ void __launch_bounds__(512, 1) k_solve_batched(SolveArgs a, BatchArgs bt)
{
    constexpr int U = 16 / CH;           // slices in flight per warp in the operator pass
    constexpr int US = CH <= 6 ? 4 : 2;  // the same with streamed tables
    constexpr int UB = 4;                // slices in flight per warp in the update pass
    __shared__ Shared sh;
    __shared__ TankState ts;
    extern __shared__ __align__(16) unsigned char dsm[];
    Grid g{a.bar, a.err, a.partials, a.budget_ns, 0u, (int)gridDim.x, 0};
    const int T = bt.T;
    // dynamic shared memory: the staged tables
    unsigned char *tdsm = dsm;
    // this CTA's tank and slices: from the planned table at first, from the
    // re-planned one (ts.tcta) once tanks have finished
    const int4 me = bt.cta[blockIdx.x];
    int tank = me.x, cend = me.w;
    Range R;
    R.s0 = me.y;
    R.s1 = me.z;
    R.warp = threadIdx.x >> 5;
    R.lane = threadIdx.x & 31;
    R.nw = blockDim.x >> 5;
    DevParams pm = bt.tprm[tank];
    int ref = pm.ref;
    float pin32 = pm.pin32;
    double pin64 = pm.pin64;
    if (threadIdx.x < 32) {
        for (int t = threadIdx.x; t < T; t += 32) {
            const int2 r = bt.tank_cta[t];
            ts.tcta[t] = r;
            ts.sfirst[t] = bt.cta[r.x].y;
            ts.nslc[t] = bt.cta[r.y - 1].z - bt.cta[r.x].y;
            ts.tend[t] = bt.cta[r.x].w;
        }
    }
    __syncwarp();  // thread 0 reads what the other lanes of warp 0 wrote
    if (threadIdx.x == 0) list_wide(ts, T);
    BTab tab = stage_btab(a.m, R, STREAM ? 0 : a.cache_cap, a.meta_slots, tdsm);  // ends with a block barrier
    // streamed tables: the ring follows the CTA's range; a range longer than
    // the metadata area (the host sizes it for every re-plan) is an error
    Ring ring{};
    if constexpr (STREAM) {
        ring = make_ring(a, R, tab.meta, tdsm, sh, CT);
        ring_retarget(ring, R.s0, tab.nmeta, tab.meta);
        if (threadIdx.x == 0 && tab.nmeta < R.s1 - R.s0) atomicCAS(a.err, 0, (int)GFM_ERR_STATE);
    }
    // every early return first lets the stages still in flight land
    auto bail = [&]() {
        if constexpr (STREAM)
            if (threadIdx.x == 0) ring_drain(ring, a.budget_ns);
        batch_abort(a, bt);
    };
    // after a re-plan: find this CTA's tank and its share of the tank's
    // slices, and stage its tables (a streamed ring is drained first and,
    // with `prefetch`, asked for the new range's first stages)
    auto take_assignment = [&](bool prefetch) {
        if constexpr (STREAM) {
            if (threadIdx.x == 0) {
                ring_drain(ring, a.budget_ns);
                if (ring.used != ring.issued) atomicCAS(a.err, 0, (int)GFM_ERR_TIMEOUT);
                ts.ring_used = ring.used;
            }
            __syncthreads();
            ring.used = ts.ring_used;
        }
        int t = 0;
        while (t < T - 1 && !(ts.tcta[t].x <= (int)blockIdx.x && (int)blockIdx.x < ts.tcta[t].y)) ++t;
        const int2 r = ts.tcta[t];
        const long long q = blockIdx.x - r.x, nq = r.y - r.x;
        tank = t;
        cend = ts.tend[t];
        R.s0 = ts.sfirst[t] + (int)((ts.nslc[t] * q) / nq);
        R.s1 = ts.sfirst[t] + (int)((ts.nslc[t] * (q + 1)) / nq);
        pm = bt.tprm[t];
        ref = pm.ref;
        pin32 = pm.pin32;
        pin64 = pm.pin64;
        tab = stage_btab(a.m, R, STREAM ? 0 : a.cache_cap, a.meta_slots, tdsm);
        if constexpr (STREAM) {
            ring_retarget(ring, R.s0, tab.nmeta, tab.meta);
            if (threadIdx.x == 0) {
                if (tab.nmeta < R.s1 - R.s0) atomicCAS(a.err, 0, (int)GFM_ERR_STATE);
                if (prefetch) ring_prefetch(ring);
            }
        }
    };
    // warp 0 counts the tanks still iterating; when some have finished,
    // every CTA re-plans the tank->CTA table and takes its new range.  Ends
    // with a CTA barrier.  (Always true: kept for the bail-out pattern.)
    auto replan_if_finished = [&]() -> bool {
        __syncthreads();
        if (threadIdx.x < 32) {
            int nact = 0;
            for (int t0 = 0; t0 < T; t0 += 32)
                nact += __popc(__ballot_sync(0xffffffffu, t0 + (int)threadIdx.x < T && ts.act[t0 + threadIdx.x] == kGo));
            if (threadIdx.x == 0) {
                ts.any_active = nact > 0;
                sh.flag = (nact > 0 && nact < ts.n_active);  // tanks finished: re-plan
                if (sh.flag) ts.n_active = nact;
            }
            __syncwarp();
            if (sh.flag) batch_rebalance(ts, T, (int)gridDim.x, false);
        }
        __syncthreads();
        if (sh.flag) {
            take_assignment(true);
            __syncthreads();
        }
        return true;
    };
    float *__restrict__ E = a.E;
    float *__restrict__ R32 = a.R32;
    float *__restrict__ S32 = a.S32;
    float *__restrict__ P32 = a.P32;
    const float *__restrict__ dinv = a.dinv32;
    const double rtol2 = a.rtol * a.rtol;
    const int cap_updates = a.max_refine + 1 + (int)(2.0 * log10(1.0 / a.rtol));

    // prologue: x0, e = 0, ||b||^2 per tank
    double vb[1] = {0.0};
    for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
        const int i = s * kSlice + R.lane;
        if (i < cend) {
            a.x64[i] = a.use_x0 ? a.p_user[a.iperm[i]] : 0.0;
            E[i] = 0.0f;
            const double bi = a.b[i];
            vb[0] += bi * bi;
        }
    }
    block_sum_f64<1>(sh, vb);
    if (!batch_allreduce<1>(g, sh, ts, bt, vb)) { bail(); return; }
    if (threadIdx.x < 32) {
        for (int t = threadIdx.x; t < T; t += 32) {
            const double bb = ts.tot[0][t];
            const double bn = (bb > 0.0) ? sqrt(bb) : 1.0;
            int ex;
            frexp(bn / sqrt((double)(a.n_per_tank ? a.n_per_tank[t] : 1)), &ex);
            ts.bnorm[t] = bn;
            ts.sc[t] = ldexp(1.0, -ex);
            ts.isc[t] = ldexp(1.0, ex);
            ts.rho_stop[t] = rtol2 * (bn * ts.sc[t]) * (bn * ts.sc[t]);
            ts.act[t] = kGo;
            ts.flag[t] = 0;
            ts.pend[t] = 0;
            ts.wait[t] = 0;
            ts.last_rep[t] = 0;
            ts.iters[t] = ts.updates[t] = ts.stall[t] = ts.last_upd[t] = ts.restarts[t] = 0;
            ts.be[t] = 0.0f;
            ts.gam_prev[t] = 1.0;
            const TankCoarse &tc = bt.tco[t];
            ts.K[t] = tc.K;
            ts.rc[t] = tc.ref_comp;
            ts.x0[t] = tc.x0;
            ts.x1[t] = tc.x1;
            for (int q = 0; q < kTankCoarse * kTankCoarse; ++q) {
                ts.Einv[q][t] = tc.Einv[q];
                ts.Einv32[q][t] = (float)tc.Einv[q];
            }
            for (int k = 0; k < kTankCoarse; ++k) {
                ts.y[k][t] = 0.0;
                ts.c32[k][t] = 0.0f;
            }
        }
    }
    __syncthreads();
    float2 *cur = a.UP0, *nxt = a.UP1;
    if (!batch_replace<CH>(a, bt, g, sh, ts, R, tank, cend, ref, pin64, cur, false, true)) {
        bail();
        return;
    }
    if (threadIdx.x < 32) {
        bool active = false;
        for (int t = threadIdx.x; t < T; t += 32) {
            const double rel2 = ts.tot[0][t] / (ts.bnorm[t] * ts.bnorm[t]);
            ts.updates[t] = 1;
            ts.best[t] = rel2;
            ts.gam[t] = ts.tot[1][t];
            ts.rho_max[t] = ts.tot[2][t];
            ts.act[t] = (rel2 <= rtol2) ? kConverged : kGo;
            active |= ts.act[t] == kGo;
        }
        active = __any_sync(0xffffffffu, active);
        if (threadIdx.x == 0) ts.any_active = active;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ts.round_age = 0;
        ts.n_active = T;  // re-plan as soon as any tank is done
        if constexpr (STREAM) ring_prefetch(ring);
    }
    if (threadIdx.x < 32) zero_bins(sh);
    // tanks that the start already solves give their CTAs away at once
    if (!replan_if_finished()) { bail(); return; }
    while (ts.any_active) {
        const bool work = ts.act[tank] == kGo && ts.wait[tank] == 0;
        const float be = ts.be[tank];
        // pass A: p = u + beta p (own and, redundantly, neighbours), s = A p, p.s,
        // and the tank's Z^T (A p) from its faces between coarse regions
        const int Kt = ts.K[tank];
        // the coarse bins were cleared by warp 0 in the last alpha step (or
        // before the loop), ahead of a CTA barrier
        FF accA[1] = {{0.f, 0.f}};
        if constexpr (STREAM) {
            // every stage is waited for, so the ring stays in step even when
            // this CTA's tank has stopped
            for (int r = 0; r < ring.nr; ++r) {
                if (ring_wait(ring, a.budget_ns)) {
                    if (work) {
                        const int sr0 = ring.s0 + r * ring.stage_slices;
                        const int sr1 = min(ring.s0 + ring.nsl, sr0 + ring.stage_slices);
                        if constexpr (CT) {
                            const StageTabCT st = ring_stage_ct(ring, r);
                            for (int sb = sr0 + R.warp; sb < sr1; sb += US * R.nw)
                                mixed_op_group<CH, US>(st, sb, sr1, R, cend, cur, P32, S32, be, ref, pin32,
                                                       ts.rc[tank], Kt, sh, accA[0]);
                        } else {
                            const StageTab st = ring_stage(ring, r);
                            for (int sb = sr0 + R.warp; sb < sr1; sb += US * R.nw)
                                mixed_op_group<CH, US>(st, sb, sr1, R, cend, cur, P32, S32, be, ref, pin32,
                                                       ts.rc[tank], Kt, sh, accA[0]);
                        }
                    }
                } else {
                    sh.ring_fail = 1;
                }
                ++ring.used;
                __syncthreads();  // stage consumed: it may be refilled
                if (sh.ring_fail) break;
                if (threadIdx.x == 0 && r + ring.n_stages < ring.nr) ring_issue(ring, r + ring.n_stages);
            }
            if (sh.ring_fail) {
                if (threadIdx.x == 0) atomicCAS(a.err, 0, (int)GFM_ERR_TIMEOUT);
                bail();
                return;
            }
            // the next pass's first stages load during the rest of the iteration
            if (threadIdx.x == 0) ring_prefetch(ring);
        }
        if (work) {
            if constexpr (!STREAM)
                for (int sb = R.s0 + R.warp; sb < R.s1; sb += U * R.nw)
                    mixed_op_group_hoisted<CH, U>(tab, sb, R.s1, R, cend, cur, P32, S32, be, ref, pin32, ts.rc[tank],
                                                  Kt, sh, accA[0]);
            if (Kt > 0) {
                // this CTA's share of the tank's cross faces
                const int2 tr = ts.tcta[tank];
                const long long q = blockIdx.x - tr.x, nq = tr.y - tr.x, span = ts.x1[tank] - ts.x0[tank];
                cross_sums_range<float>(a.cross, ts.x0[tank] + (int)(span * q / nq),
                                        ts.x0[tank] + (int)(span * (q + 1) / nq), Kt, sh.zbw32,
                                        [&](const CrossFace &cf) {
                                            const float2 vo = cur[cf.o], vv = cur[cf.v];
                                            return cf.g32 * (fmaf(be, vo.y, vo.x) - fmaf(be, vv.y, vv.x));
                                        });
            }
        }
        float2 blkA[1 + kTankCoarse];
        {
            float2 b1[1];
            block_sum_ff2<1>(sh, accA, b1);
            blkA[0] = b1[0];
        }
        if (work && Kt > 0 && threadIdx.x < 32) finish_bins<float>(sh.zbw32, sh.zpin32, ts.rc[tank], Kt, R.nw, sh.zb32);
        for (int k = 0; k < kTankCoarse; ++k) blkA[1 + k] = make_float2((work && k < Kt) ? sh.zb32[k] : 0.0f, 0.0f);
        if (!batch_allreduce_ff<1 + kTankCoarse>(g, sh, ts, bt, blkA)) { bail(); return; }
        if (threadIdx.x < 32) {
            zero_bins(sh);  // this pass's bins were read before the all-reduce
            for (int t = threadIdx.x; t < T; t += 32) {
                if (ts.act[t] != kGo || ts.wait[t]) continue;
                const double ps = ts.tot[0][t];
                const bool ok = ps > 0.0 && isfinite(ps) && ts.gam[t] > 0.0;
                // alpha in FP32, the vectors' precision (an FP64 divide per tank
                // costs more than the whole step on GB300's FP64 pipe)
                const float al = ok ? (float)ts.gam[t] / (float)ps : 0.0f;
                ts.al[t] = al;
                ts.flag[t] = ok ? 0 : kRestart;
                if (ok && ts.K[t] > 0) {  // y -= alpha Z^T A p (FP64), c = E^{-1} y (FP32)
                    for (int k = 0; k < ts.K[t]; ++k) ts.y[k][t] = fma(-(double)al, ts.tot[1 + k][t], ts.y[k][t]);
                    tank_coarse_solve32(ts, t);
                }
            }
        }
        __syncthreads();
        const float al = ts.al[tank];
        // pass B: e += alpha p, r -= alpha s, u = D^{-1} r; r.u, r.r
        FF accB[2] = {{0.f, 0.f}, {0.f, 0.f}};
        if (work && ts.flag[tank] == 0) {
            for (int sb = R.s0 + R.warp; sb < R.s1; sb += UB * R.nw) {
                int ii[UB], cm[UB];
                bool act[UB];
                float pi[UB], si[UB], ri[UB], ei[UB], di[UB];
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    ii[u] = (sb + u * R.nw) * kSlice + R.lane;
                    act[u] = sb + u * R.nw < R.s1 && ii[u] < cend;
                    // every load of the group in flight together
                    pi[u] = act[u] ? __ldcs(P32 + ii[u]) : 0.f;
                    si[u] = act[u] ? __ldcs(S32 + ii[u]) : 0.f;
                    ri[u] = act[u] ? __ldcs(R32 + ii[u]) : 0.f;
                    ei[u] = act[u] ? __ldcs(E + ii[u]) : 0.f;
                    di[u] = act[u] ? __ldcs(dinv + ii[u]) : 0.f;
                    cm[u] = (act[u] && Kt > 0) ? (int)a.comp[ii[u]] : -1;
                }
#pragma unroll
                for (int u = 0; u < UB; ++u) {
                    if (act[u]) {
                        __stcs(E + ii[u], fmaf(al, pi[u], ei[u]));
                        const float rn = fmaf(-al, si[u], ri[u]);
                        __stcs(R32 + ii[u], rn);
                        float un = rn * di[u];
                        if (cm[u] >= 0) un += ts.c32[cm[u]][tank];
                        nxt[ii[u]] = make_float2(un, pi[u]);
                        ff_add(accB[0], rn * un);
                        ff_add(accB[1], rn * rn);
                    }
                }
            }
        } else if (ts.act[tank] == kGo && ts.wait[tank]) {
            // an idle tank keeps its (u, p) pairs across the buffer swap
            for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
                const int i = s * kSlice + R.lane;
                if (i < cend) nxt[i] = cur[i];
            }
        }
        float2 blkB[2];
        block_sum_ff2<2>(sh, accB, blkB);
        if (!batch_allreduce_ff<2>(g, sh, ts, bt, blkB)) { bail(); return; }
        { float2 *tmp = cur; cur = nxt; nxt = tmp; }  // cur = (u_new, p)
        // Replacements come in rounds.  A tank that asks for one because its
        // FP32 residual fell a decade or 1000 iterations passed keeps
        // iterating until the next round, which comes once every
        // kReplaceRound iterations while any tank waits.  A tank whose FP32
        // residual claims convergence, or fell its decade within two rounds
        // of its last replacement, stops and idles until then: its FP32
        // recurrence would run on past convergence (a tank of a few dozen
        // cells does in a handful of iterations) and the direction kept
        // through the replacement would be noise, which stalls the
        // refinement.  The round comes at once when a tank cannot go on
        // (breakdown, iteration cap) or no tank is left iterating.  Every
        // replacement holds all CTAs at its barriers, so serving many tanks
        // at one of them costs the others far less; a wait of kReplaceRound
        // iterations moves an FP32 residual by about a decade at most on
        // these systems, well inside what FP32 resolves.
        if (threadIdx.x < 32) {
            bool now = false, waiting = false, going = false;
            for (int t = threadIdx.x; t < T; t += 32) {
                if (ts.act[t] != kGo) continue;
                if (ts.wait[t]) { waiting = true; continue; }
                if (ts.flag[t] == kRestart) { now = true; continue; }
                const int it = ++ts.iters[t];
                ts.gam_prev[t] = ts.gam[t];
                const double gam = ts.tot[0][t], rho = ts.tot[1][t];
                ts.gam[t] = gam;
                if (rho > ts.rho_max[t]) ts.rho_max[t] = rho;
                if (it >= a.max_iters) {
                    ts.flag[t] = kNotConverged;
                    now = true;
                } else if (!(gam > 0.0)) {
                    ts.flag[t] = kUpdate;
                    ts.last_upd[t] = it;
                    now = true;
                } else if (rho <= ts.rho_stop[t]) {
                    ts.pend[t] = kUpdate;
                    ts.wait[t] = 1;
                    ts.last_upd[t] = it;
                } else {
                    if (ts.pend[t] == 0 && (rho <= 1e-2 * ts.rho_max[t] || it - ts.last_upd[t] >= 1000)) {
                        ts.pend[t] = kUpdate;
                        ts.last_upd[t] = it;
                        if (it - ts.last_rep[t] < 2 * kReplaceRound) ts.wait[t] = 1;
                    }
                    if (ts.wait[t] == 0) {
                        ts.be[t] = (float)gam / (float)ts.gam_prev[t];
                        going = true;
                    }
                }
                waiting |= ts.pend[t] != 0;
            }
            going = __any_sync(0xffffffffu, going);
            now = now || (waiting && !going);
            now = __any_sync(0xffffffffu, now);
            waiting = __any_sync(0xffffffffu, waiting);
            if (threadIdx.x == 0) {
                ++ts.round_age;
                ts.any_flag = now || (waiting && ts.round_age >= kReplaceRound);
            }
            __syncwarp();
            if (ts.any_flag) {
                for (int t = threadIdx.x; t < T; t += 32)
                    if (ts.act[t] == kGo && ts.flag[t] == 0) ts.flag[t] = ts.pend[t];
                if (threadIdx.x == 0) ts.round_age = 0;
            }
        }
        __syncthreads();
        if (ts.any_flag) {
            // fold e into x and replace r by the true residual for the tanks
            // that asked (restarts also clear their direction)
            if (!batch_replace<CH>(a, bt, g, sh, ts, R, tank, cend, ref, pin64, cur, true, false)) {
                bail();
                return;
            }
            if (threadIdx.x < 32) {
                for (int t = threadIdx.x; t < T; t += 32) {
                    const int f = ts.flag[t];
                    if (ts.act[t] != kGo || f == 0) continue;
                    ts.flag[t] = 0;
                    ts.pend[t] = 0;
                    ts.wait[t] = 0;
                    ts.last_rep[t] = ts.iters[t];
                    ++ts.updates[t];
                    const double rel2 = ts.tot[0][t] / (ts.bnorm[t] * ts.bnorm[t]);
                    if (rel2 <= rtol2) { ts.act[t] = kConverged; continue; }
                    if (f == kNotConverged) { ts.act[t] = kNotConverged; continue; }
                    if (f == kRestart) {
                        if (++ts.restarts[t] > 3) { ts.act[t] = kBreakdown; continue; }
                    } else {
                        if (rel2 < 0.25 * ts.best[t]) { ts.best[t] = rel2; ts.stall[t] = 0; }
                        else ++ts.stall[t];
                    }
                    if (ts.stall[t] > 8 || ts.updates[t] > cap_updates) { ts.act[t] = kNotConverged; continue; }
                    ts.gam[t] = ts.tot[1][t];
                    ts.rho_max[t] = ts.tot[2][t];
                    ts.be[t] = (f == kRestart || !(ts.gam_prev[t] > 0.0)) ? 0.0f
                                                                           : (float)ts.gam[t] / (float)ts.gam_prev[t];
                }
            }
            // tanks only finish in a replacement round: re-plan here
            if (!replan_if_finished()) { bail(); return; }
        }
    }
    // every tank gets CTAs again for the final residuals
    if (threadIdx.x < 32) batch_rebalance(ts, T, (int)gridDim.x, true);
    __syncthreads();
    take_assignment(false);
    // per-tank finish: true residual, solution in caller order, L1 residual
    if (!grid_sync(g, sh)) { bail(); return; }
    double v[2] = {0.0, 0.0};
    for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
        const int i = s * kSlice + R.lane;
        if (i < cend) {
            const double xi = a.x64[i];
            const double r = a.b[i] - apply64_diff<CH>(a.m, row_of(a.m, s), R.lane, a.x64, xi, i == ref ? pin64 : 0.0);
            a.r64[i] = r;
            v[0] += r * r;
            v[1] += xi;
        }
    }
    block_sum_f64<2>(sh, v);
    if (!batch_allreduce<2>(g, sh, ts, bt, v)) { bail(); return; }
    if (threadIdx.x < 32) {
        for (int t = threadIdx.x; t < T; t += 32) {
            ts.xavg[t] = ts.tot[1][t] / (double)(a.n_per_tank ? a.n_per_tank[t] : 1);
            ts.best[t] = ts.tot[0][t];  // ||r||^2, kept for the record
        }
    }
    __syncthreads();
    const double xavg = ts.xavg[tank];
    double w[2] = {0.0, 0.0};
    for (int s = R.s0 + R.warp; s < R.s1; s += R.nw) {
        const int i = s * kSlice + R.lane;
        if (i < cend) {
            const double xi = a.x64[i];
            a.p_user[a.iperm[i]] = xi;
            const double r = a.r64[i];
            const double rs = (i == ref) ? pin64 : 0.0;
            const double Ax = a.b[i] - r;
            w[0] += fabs(r);
            w[1] += fabs(Ax - xavg * rs) + fabs(a.b[i] - xavg * rs);
        }
    }
    block_sum_f64<2>(sh, w);
    if (!batch_allreduce<2>(g, sh, ts, bt, w)) { bail(); return; }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const int e = ld_volatile_i32(a.err);
        for (int t = threadIdx.x; t < T; t += 32) {
            int st = GFM_OK;
            if (ts.act[t] == kNotConverged) st = GFM_ERR_NOT_CONVERGED;
            else if (ts.act[t] == kBreakdown) st = GFM_ERR_BREAKDOWN;
            if (e != 0) st = e;
            bt.infos[t].iters = ts.iters[t];
            bt.infos[t].refinements = ts.updates[t];
            bt.infos[t].status = st;
            bt.infos[t].reserved = 0;
            bt.infos[t].rel_res_l2 = sqrt(ts.best[t]) / ts.bnorm[t];
            bt.infos[t].rel_res_l1 = ts.tot[0][t] / (ts.tot[1][t] + 1e-300);
        }
    }
}

const void *batched_kernel(int max_width, bool streamed, bool compact)
{
    if (max_width <= 4) {
        if (streamed && compact) return (const void *)k_solve_batched<4, true, true>;
        return streamed ? (const void *)k_solve_batched<4, true> : (const void *)k_solve_batched<4, false>;
    }
    if (streamed && compact) return (const void *)k_solve_batched<8, true, true>;
    return streamed ? (const void *)k_solve_batched<8, true> : (const void *)k_solve_batched<8, false>;
}

// Instantiations by faces per row chunk (4 for 2D hex meshes, 8 otherwise)
// and, for the mixed solver, by how the operator pass reads the tables
// (streamed through shared-memory stages -- in full or compact form -- or
// cached / read in place).
const void *solver_kernel(Mode m, int max_width, int threads, bool streamed, bool compact, bool fused)
{
    (void)threads;
    const bool ct = streamed && compact;
    if (m == Mode::MIXED && fused && !ct) {
        if (max_width <= 4) return streamed ? (const void *)k_solve_fused<4, true> : (const void *)k_solve_fused<4, false>;
        if (streamed && max_width <= 6) return (const void *)k_solve_fused<6, true>;
        return streamed ? (const void *)k_solve_fused<8, true> : (const void *)k_solve_fused<8, false>;
    }
    if (max_width <= 4) {
        if (m == Mode::FP64) return (const void *)k_solve_fp64<4>;
        if (ct) return (const void *)k_solve_mixed<4, true, true>;
        return streamed ? (const void *)k_solve_mixed<4, true> : (const void *)k_solve_mixed<4, false>;
    }
    if (m == Mode::FP64) return (const void *)k_solve_fp64<8>;
    if (streamed && max_width <= 6) {  // hexahedra
        if (ct) return (const void *)k_solve_mixed<6, true, true>;
        return (const void *)k_solve_mixed<6, true>;
    }
    if (ct) return (const void *)k_solve_mixed<8, true, true>;
    return streamed ? (const void *)k_solve_mixed<8, true> : (const void *)k_solve_mixed<8, false>;
}

int solver_max_threads() { return 512; }

}  // namespace gfm
