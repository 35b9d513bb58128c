// gfm_solve_csr_noalloc: FP64 Jacobi-PCG of a caller-held CSR system that
// allocates no device memory.
//
// Who needs it: code that runs inside a host program owning the device
// memory -- a CFD code or plugin whose memory comes from the host's pool or
// sits under a hard memory cap, where a cudaMalloc would be refused or would
// fragment the pool -- and time-critical loops in which cudaMalloc/cudaFree
// are off limits because they can synchronise the whole device.  Such a
// caller passes its own device arrays; every temporary the solve needs (the
// CG vectors, the per-CTA partial sums, the grid-barrier counter) lives in
// the file-scope array below, which the CUDA runtime places when it loads
// this library's device code on a GPU and keeps there until the process
// exits.
//
// The kernel is a variant of the handle-based FP64 persistent solver: the
// same Jacobi-preconditioned CG with deterministic grid reductions, bounded
// grid barriers and restarts from the true residual, reading a CSR matrix
// from the caller instead of the handle's sliced-ELL tables, one thread per
// row.  All calls on a device share the one array, which keeps the last
// call's contents; the barrier block is cleared at every call, and every
// other word is written before it is read.  Two calls whose kernels overlap
// on the GPU (different streams, or different host threads) race on the
// array and corrupt each other's results: order them on one stream.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "gfm.h"

namespace {

constexpr int kMaxCells = GFM_NOALLOC_MAX_CELLS;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxGrid = 1024;
constexpr int kNR = 3;          // values per grid reduction
constexpr int kMaxChecks = 30;  // true-residual restarts per call
constexpr int kMaxDevices = 256;

// Layout of the scratch array, in doubles.
constexpr size_t kCtl = 0;                                      // [32]: barrier counter (u64), error flag (int)
constexpr size_t kPart = 32;                                    // [2][kNR][kMaxGrid] per-CTA partial sums
constexpr size_t kVec = kPart + 2 * (size_t)kNR * kMaxGrid;     // r, p, q, dinv: [kMaxCells] each
constexpr size_t kScratchDoubles = kVec + 4 * (size_t)kMaxCells;  // 8.05 MiB at 262144 cells

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

struct Args {
    int n, nnz;
    const int *rp, *col;
    const double *val, *b;
    double *x;
    double rtol;
    int max_iters, use_x0, G;
    unsigned long long budget_ns;
    gfm_solve_info *info;
    double *scr;
};

struct Bar {
    unsigned long long *count;
    int *err;
    double *part;
    unsigned long long budget, epoch;
    int G, parity;
};

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void add_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier on a monotone 64-bit arrival counter.  Every wait is bounded:
// past the budget the CTA records GFM_ERR_TIMEOUT and all CTAs return.
// False means the solve must stop (timeout, or an error any CTA recorded).
__device__ bool bar_sync(Bar &g, int &flag)
{
    __syncthreads();
    g.epoch += 1;
    if (threadIdx.x == 0) {
        int fail = 0;
        __threadfence();
        add_release(g.count, 1ull);
        const unsigned long long target = g.epoch * (unsigned long long)g.G;
        const unsigned long long t0 = now_ns();
        while (load_acquire(g.count) < target) {
            if (*(volatile int *)g.err != 0) { fail = 1; break; }
            if (now_ns() - t0 > g.budget) {
                atomicCAS(g.err, 0, (int)GFM_ERR_TIMEOUT);
                fail = 1;
                break;
            }
        }
        __threadfence();
        if (*(volatile int *)g.err != 0) fail = 1;
        flag = fail;
    }
    __syncthreads();
    return flag == 0;
}

// Sum of `nr` per-thread values over the whole grid, bitwise identical in
// every CTA: fixed-order block sums, then each CTA adds all CTAs' partials in
// the same order.
template <int NR>
__device__ bool grid_sum(Bar &g, double (&red)[kWarps][kNR], double (&tot)[kNR], int &flag, double (&v)[NR])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
        g.part[((size_t)g.parity * kNR + threadIdx.x) * kMaxGrid + blockIdx.x] = s;
    }
    if (!bar_sync(g, flag)) return false;
    if (warp < NR) {
        const double *src = g.part + ((size_t)g.parity * kNR + warp) * kMaxGrid;
        double s = 0.0;
        for (int c = lane; c < g.G; c += 32) s += __ldcg(src + c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) tot[warp] = s;
    }
    g.parity ^= 1;
    __syncthreads();
    return true;
}

__device__ __forceinline__ double row_dot(const Args &a, int i, const double *v)
{
    double s = 0.0;
    const int e1 = a.rp[i + 1];
    for (int e = a.rp[i]; e < e1; ++e) s += a.val[e] * v[a.col[e]];
    return s;
}

__device__ void write_info(const Args &a, int iters, int checks, int status, double l2, double l1)
{
    if (a.info == nullptr || blockIdx.x != 0 || threadIdx.x != 0) return;
    a.info->iters = iters;
    a.info->refinements = checks;
    a.info->status = status;
    a.info->reserved = 0;
    a.info->rel_res_l2 = l2;
    a.info->rel_res_l1 = l1;
}

__global__ void __launch_bounds__(kThreads) k_pcg_csr_noalloc(Args a)
{
    __shared__ double red[kWarps][kNR];
    __shared__ double tot[kNR];
    __shared__ int flag;
    Bar g{reinterpret_cast<unsigned long long *>(a.scr + kCtl), reinterpret_cast<int *>(a.scr + kCtl + 1),
          a.scr + kPart, a.budget_ns, 0ull, a.G, 0};
    double *r = a.scr + kVec, *p = r + kMaxCells, *q = p + kMaxCells, *dinv = q + kMaxCells;
    const int n = a.n;
    const int i0 = blockIdx.x * kThreads + threadIdx.x, stride = a.G * kThreads;
    const double rtol2 = a.rtol * a.rtol;
    int iters = 0, checks = 0, status = GFM_ERR_NOT_CONVERGED;

    // Validate the caller's CSR structure before any vector is gathered
    // through it: 0 <= row_ptr[i] <= row_ptr[i+1] <= nnz and 0 <= col < n.
    // A row with bad bounds is skipped, so the check itself reads only
    // row_ptr [n+1] and, within checked bounds, col/val [nnz].  Jacobi
    // weights from the diagonal entries; a row without a positive one is an
    // argument error too.  Start vector.  Every row is checked by some CTA
    // before the barrier, and any error stops every CTA after it.
    int bad = 0;
    for (int i = i0; i < n; i += stride) {
        const int e0 = a.rp[i], e1 = a.rp[i + 1];
        double d = 0.0;
        if (e0 < 0 || e1 < e0 || e1 > a.nnz) {
            bad = 1;
        } else {
            for (int e = e0; e < e1; ++e) {
                const int c = a.col[e];
                if (c < 0 || c >= n) bad = 1;
                else if (c == i) d += a.val[e];
            }
        }
        if (!(d > 0.0) || !isfinite(d)) bad = 1;
        dinv[i] = 1.0 / d;
        if (!a.use_x0) a.x[i] = 0.0;
    }
    if (bad) atomicCAS(g.err, 0, (int)GFM_ERR_ARG);
    if (!bar_sync(g, flag)) goto abort;

    for (;;) {
        // restart from the true residual r = b - A x, p = D^{-1} r
        double v[3] = {0.0, 0.0, 0.0};
        for (int i = i0; i < n; i += stride) {
            const double ri = a.b[i] - row_dot(a, i, a.x);
            const double zi = dinv[i] * ri;
            r[i] = ri;
            p[i] = zi;
            v[0] += ri * ri;
            v[1] += ri * zi;
            v[2] += a.b[i] * a.b[i];
        }
        if (!grid_sum<3>(g, red, tot, flag, v)) goto abort;
        ++checks;
        const double bb = tot[2];
        double rz = tot[1];
        if (bb == 0.0) {  // b = 0: the solution is p = 0
            for (int i = i0; i < n; i += stride) a.x[i] = 0.0;
            status = GFM_OK;
            break;
        }
        if (!isfinite(tot[0])) { status = GFM_ERR_BREAKDOWN; break; }
        if (tot[0] <= rtol2 * bb) { status = GFM_OK; break; }
        if (iters >= a.max_iters || checks > kMaxChecks) break;

        for (;;) {
            double w[1] = {0.0};
            for (int i = i0; i < n; i += stride) {
                const double qi = row_dot(a, i, p);
                q[i] = qi;
                w[0] += p[i] * qi;
            }
            if (!grid_sum<1>(g, red, tot, flag, w)) goto abort;
            const double pq = tot[0];
            if (!(pq > 0.0) || !isfinite(pq)) { status = GFM_ERR_BREAKDOWN; goto done; }
            const double alpha = rz / pq;
            double u[2] = {0.0, 0.0};
            for (int i = i0; i < n; i += stride) {
                a.x[i] += alpha * p[i];
                const double ri = r[i] - alpha * q[i];
                r[i] = ri;
                u[0] += ri * ri;
                u[1] += ri * (dinv[i] * ri);
            }
            if (!grid_sum<2>(g, red, tot, flag, u)) goto abort;
            ++iters;
            if (tot[0] <= rtol2 * bb || iters >= a.max_iters) break;  // verify on the true residual
            const double beta = tot[1] / rz;
            rz = tot[1];
            for (int i = i0; i < n; i += stride) p[i] = dinv[i] * r[i] + beta * p[i];
            if (!bar_sync(g, flag)) goto abort;
        }
    }

done:
    // final record: true residual (L2, and the normalised L1 residual with
    // the row sums of A applied to the mean of x)
    {
        if (!bar_sync(g, flag)) goto abort;
        double v[3] = {0.0, 0.0, 0.0};
        for (int i = i0; i < n; i += stride) {
            const double ri = a.b[i] - row_dot(a, i, a.x);
            r[i] = ri;
            v[0] += ri * ri;
            v[1] += a.x[i];
            v[2] += a.b[i] * a.b[i];
        }
        if (!grid_sum<3>(g, red, tot, flag, v)) goto abort;
        const double rr = tot[0], xavg = tot[1] / (double)n, bb = tot[2];
        double w[2] = {0.0, 0.0};
        for (int i = i0; i < n; i += stride) {
            double rs = 0.0;
            for (int e = a.rp[i]; e < a.rp[i + 1]; ++e) rs += a.val[e];
            const double ax = a.b[i] - r[i];
            w[0] += fabs(r[i]);
            w[1] += fabs(ax - xavg * rs) + fabs(a.b[i] - xavg * rs);
        }
        if (!grid_sum<2>(g, red, tot, flag, w)) goto abort;
        write_info(a, iters, checks, status, bb > 0.0 ? sqrt(rr / bb) : 0.0, tot[0] / (tot[1] + 1e-300));
        return;
    }

abort:
    write_info(a, iters, checks, *(volatile int *)g.err, -1.0, -1.0);
}

struct DeviceScratch {
    double *ptr = nullptr;
    int grid_cap = 0;
};

std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];

// One-time set-up on the current device: the device address of the scratch
// array (this also loads the device code if the runtime loads it lazily) and
// the largest co-resident grid.
gfm_status setup_current_device(DeviceScratch &out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GFM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return GFM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch &d = g_dev[dev];
    if (d.ptr == nullptr) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return GFM_ERR_CUDA;
        int coop = 0, sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
            return GFM_ERR_CUDA;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GFM_ERR_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_csr_noalloc, kThreads, 0) != cudaSuccess ||
            per_sm < 1)
            return GFM_ERR_CUDA;
        d.grid_cap = sms * per_sm < kMaxGrid ? sms * per_sm : kMaxGrid;
        d.ptr = static_cast<double *>(ptr);
    }
    out = d;
    return GFM_OK;
}

}  // namespace

extern "C" gfm_status gfm_solve_csr_noalloc(int32_t n, int32_t nnz, const int32_t *row_ptr, const int32_t *col,
                                            const double *val, const double *b, double *x, double rtol,
                                            int32_t max_iters, int32_t use_x0, double timeout_ms,
                                            gfm_solve_info *info, gfm_stream stream)
{
    if (n < 1 || n > kMaxCells) return GFM_ERR_ARG;  // beyond the fixed scratch capacity
    if (nnz < n) return GFM_ERR_ARG;                  // every row needs its diagonal entry
    if (!row_ptr || !col || !val || !b || !x) return GFM_ERR_ARG;
    if (!(rtol > 0.0) || !std::isfinite(rtol) || max_iters < 0 || !(timeout_ms > 0.0) || !std::isfinite(timeout_ms))
        return GFM_ERR_ARG;
    (void)cudaGetLastError();  // a non-sticky error left by earlier, unrelated work
    DeviceScratch d;
    const gfm_status st = setup_current_device(d);
    if (st != GFM_OK) return st;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int want = (n + kThreads - 1) / kThreads;
    Args a;
    a.n = n;
    a.nnz = nnz;
    a.rp = row_ptr;
    a.col = col;
    a.val = val;
    a.b = b;
    a.x = x;
    a.rtol = rtol;
    a.max_iters = max_iters;
    a.use_x0 = use_x0 ? 1 : 0;
    a.G = want < d.grid_cap ? want : d.grid_cap;
    const double ns = timeout_ms * 1e6;
    a.budget_ns = ns > 1.8e19 ? 18000000000000000000ull : (unsigned long long)ns;
    a.info = info;
    a.scr = d.ptr;
    if (cudaMemsetAsync(d.ptr + kCtl, 0, 32 * sizeof(double), s) != cudaSuccess) return GFM_ERR_CUDA;
    void *args[] = {&a};
    if (cudaLaunchCooperativeKernel((const void *)k_pcg_csr_noalloc, dim3(a.G), dim3(kThreads), args, 0, s) !=
        cudaSuccess)
        return GFM_ERR_CUDA;
    return GFM_OK;
}
