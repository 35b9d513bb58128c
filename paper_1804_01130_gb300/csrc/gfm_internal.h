// Internal declarations shared by the libgfm translation units (host + device).
// Not part of the public ABI (include/gfm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfm.h"

namespace gfm {

constexpr int kSlice = 32;  // cells per sliced-ELL slice (one warp, one lane per cell)

// Written on the device by the assembly, read by the solver kernels, so that
// assembling and solving need no host round trip.
struct DevParams {
    double pin64;   // diagonal of the pinned cell before pinning (0 = no pin)
    float pin32;    // (float)pin64
    int32_t ref;    // internal index of the pinned cell, -1 = none
    double bsum;    // sum of b (compatibility of an unpinned system)
    double babs;    // sum of |b|
};

// Sliced-ELL cell-to-face table in the internal (renumbered) cell order.
// Slot k of the cell in lane l of slice s is at slice_ptr[s] + k*32 + l.
// Slots of a cell are sorted by ascending caller face index; padding slots
// have face == 0, col == the cell itself and zero coefficients.
struct Sell {
    int32_t n;           // cells
    int32_t n_pad;       // n rounded up to a multiple of 32
    int32_t n_slices;
    int32_t n_slots;
    const int32_t *slice_ptr;  // [n_slices + 1]
    const int32_t *col;        // [n_slots] internal index of the other cell
    const int32_t *face;       // [n_slots] +(f+1) if the cell owns face f, -(f+1) if neighbour, 0 pad
    double *val64;             // [n_slots] gamma_f   (FP64)
    float *val32;              // [n_slots] (float)gamma_f
};

// Everything a persistent solver kernel needs.  Vectors are in internal order
// and padded to n_pad.
struct SolveArgs {
    Sell m;
    const DevParams *prm;
    const double *b;       // right-hand side (internal order)
    const double *diag64;  // diag incl. pin (internal order)
    const double *dinv64;  // 1/diag
    double *x64;           // iterate (FP64)
    double *r64;           // residual (FP64)
    double *p64, *q64;     // FP64-mode CG vectors
    float2 *UP0, *UP1;     // MIXED: (u, p) pairs, double-buffered (gathered)
    float *R32, *S32, *E;  // MIXED: scaled residual, s = A p, FP32 correction
    const float *dinv32;   // MIXED: 1 / (float)diag
    const int32_t *iperm;  // [n] internal -> caller index
    double *p_user;        // caller-order x0 in / solution out
    double rtol, inner_rtol;
    int32_t max_iters, max_refine, use_x0;
    unsigned long long budget_ns;
    unsigned int *bar;     // grid-barrier arrival counter (zeroed before launch)
    int *err;              // device status (zeroed before launch)
    double *partials;      // [2][grid][4] per-CTA partial sums
    gfm_solve_info *info;  // device-side result
};

// ---- assembly (gfm_assemble.cu) -----------------------------------------
struct FaceArgs {
    int32_t n, F;
    const int32_t *owner, *neighbour;
    const double *Sf, *C;
    const double *alpha, *phi;
    double rho_w, rho_a, g0, g1, g2;
    double *lambda, *gamma, *jump, *sigma;
    int8_t *kind;
};
cudaError_t launch_faces(const FaceArgs &a, cudaStream_t s);

struct CellArgs {
    Sell m;
    const double *gamma, *sigma;
    int32_t ref;  // internal index of the pinned cell, -1 none
    double ref_value;
    double *b, *diag, *dinv;
    float *dinv32;
    DevParams *prm;
};
cudaError_t launch_cells(const CellArgs &a, cudaStream_t s);
cudaError_t launch_bsums(const double *b, int32_t n, DevParams *prm, cudaStream_t s);

cudaError_t launch_corrected_flux(int32_t F, const int32_t *owner, const int32_t *neighbour, const double *gamma,
                                  const double *jump, const double *phi, const double *p, double *out,
                                  cudaStream_t s);

struct AdjointArgs {
    int32_t n, F;
    const int32_t *owner, *neighbour;
    const double *C, *alpha, *lambda, *gamma, *jump;
    const int8_t *kind;
    double rho_w, rho_a, g0, g1, g2;
    const double *p, *mu;  // caller order
    double *dL_dphi, *dL_dlam;
    Sell m;
    const int32_t *perm;   // caller -> internal
    const int32_t *iperm;  // internal -> caller
    double *dL_dalpha;     // caller order
};
cudaError_t launch_adjoint_faces(const AdjointArgs &a, cudaStream_t s);
cudaError_t launch_adjoint_cells(const AdjointArgs &a, cudaStream_t s);

cudaError_t launch_gather(const double *src_user, const int32_t *iperm, double *dst_internal, int32_t n,
                          int32_t n_pad, cudaStream_t s);

// ---- solver (gfm_solve.cu) ----------------------------------------------
enum class Mode { FP64 = 0, MIXED = 1 };
const void *solver_kernel(Mode m, int max_width, int threads);
int solver_max_threads();

}  // namespace gfm
