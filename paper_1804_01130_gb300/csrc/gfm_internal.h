// Internal declarations shared by the libgfm translation units (host + device).
// Not part of the public ABI (include/gfm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfm.h"

namespace gfm {

constexpr int kSlice = 32;  // cells per sliced-ELL slice (one warp, one lane per cell)
constexpr int kMaxCoarse = 8;         // coarse vectors of the two-level preconditioner
constexpr int kMaxCandidates = 4096;  // components examined when choosing them
constexpr int kMaxTanks = 128;        // tanks of one batched solve
constexpr int kMaxStages = 4;         // shared-memory stages of streamed slice tables
constexpr int kCoarseEParts = 128;    // blocks summing E = Z^T A Z

// Physics of one tank of a batch (device copy of gfm_phys, ref internal).
struct TankPhys {
    double rho_w, rho_a, g0, g1, g2, ref_value;
    int32_t ref;  // internal index of the pinned cell, -1 = none
    int32_t pad;
};

// Two-level preconditioner data, rebuilt by every assembly.  The coarse space
// is spanned by the indicator vectors of the largest connected regions of one
// phase (cells joined by non-interface faces); E = Z^T A Z and its inverse.
// Faces whose two cells lie in different coarse regions (or one in none) are
// listed so that Z^T (A v) can be formed from them exactly.
struct Coarse {
    int32_t K;       // coarse vectors in use (0 = Jacobi only)
    int32_t n_cand;  // regions of at least min_size cells
    int32_t n_cross; // listed cross faces
    int32_t ref_comp;  // coarse region of the pinned cell, -1 = none
    int32_t roots[kMaxCoarse];
    int32_t sizes[kMaxCoarse];
    double E[kMaxCoarse * kMaxCoarse];
    double Einv[kMaxCoarse * kMaxCoarse];
};

// Coarse space of one tank of a batch: its up-to-kTankCoarse largest
// one-phase regions (typically the water body and the air above it), E =
// Z^T A Z of those regions and its inverse, and the tank's stretch
// [x0, x1) of the face-ordered cross-face list.
constexpr int kTankCoarse = 2;
constexpr int kMaxReduce = 16;  // most values one grid all-reduce of a single mesh sums
constexpr int kBatchNR = 3 + kTankCoarse;  // most values one batched all-reduce sums
constexpr int kLaneSum = 8;                // tanks with more CTAs are summed by a warp
struct TankCoarse {
    int32_t K, ref_comp, x0, x1;
    int32_t roots[kTankCoarse], sizes[kTankCoarse];
    double E[kTankCoarse * kTankCoarse];
    double Einv[kTankCoarse * kTankCoarse];
};

// One face between two coarse regions: internal cell indices, coefficient,
// and the regions (a of cell o, b of cell v; -1 = not in a coarse region).
struct CrossFace {
    int32_t o, v;
    int8_t a, b;
    float g32;
    double g64;
};

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
    // Compact form of the same table for the streamed mixed operator pass
    // (nullptr when unused): per slot (value code << 16) | (uint16)(col - i),
    // i the slot's own cell; a code indexes dict, kEscape means "read val32".
    const uint32_t *ent;       // [n_slots]
    const float *dict;         // [n_dict] FP32 coefficients; the last one is 0 (padding)
    int32_t n_dict;
};

constexpr uint32_t kEscape = 0xFFFFu;  // compact-table code: coefficient not in the dictionary
constexpr int kMaxDict = 4096;         // dictionary entries (FP32), staged in shared memory

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
    float *P32;            // MIXED: this iteration's direction p (written whole, read by the update pass)
    float4 *Q0, *Q1;       // MIXED, fused form: (q, t, p, region) per cell, double-buffered (gathered)
    const float *dinv32;   // MIXED: 1 / (float)diag
    const int32_t *iperm;  // [n] internal -> caller index
    double *p_user;        // caller-order x0 in / solution out
    double rtol, inner_rtol;
    int32_t max_iters, max_refine, use_x0;
    unsigned long long budget_ns;
    const Coarse *coarse;  // two-level preconditioner (K = 0: Jacobi only)
    const int8_t *comp;    // [n_pad] coarse region of each internal cell, -1 none
    const CrossFace *cross;  // [coarse->n_cross]
    const int32_t *n_per_tank;  // batched: real cells of each tank (else nullptr)
    int32_t cache_cap;     // slots of a CTA's slice tables staged in shared memory
    int32_t meta_slots;    // slice-metadata entries reserved in shared memory
    int32_t n_stages;      // MIXED: > 0 = the operator pass streams the tables through
                           // this many shared-memory stages (bulk async copies)
    int32_t stage_slices;  // slices per stage (a multiple of the slices a pass round covers)
    int32_t stage_cap;     // slots per stage
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
    const int32_t *ftank;    // batched: tank of each face (else nullptr)
    const TankPhys *tphys;   // batched: physics per tank
    const double *rau;       // face Rhie-Chow coefficient 1/a_P (nullptr = 1)
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
    const int32_t *iperm;    // internal -> caller (-1 on padding cells)
    const int32_t *stank;    // batched: tank of each slice (else nullptr)
    const TankPhys *tphys;   // batched: ref cell and value per tank
    DevParams *tprm;         // batched: pin per tank
    // compact table (nullptr = not written): codes from the face's kind and
    // geometric class (2 cls for a wet face, 2 cls + 1 for a dry one)
    uint32_t *ent;
    const int32_t *fcls;
    const int8_t *kind;
    int32_t pad_code;
};
cudaError_t launch_cells(const CellArgs &a, cudaStream_t s);

// sigma = phi + gamma J for a new predicted flux (coefficients unchanged)
cudaError_t launch_sigma(int32_t F, const double *phi, const double *gamma, const double *jump, double *sigma,
                         cudaStream_t s);

// c_f = (S.S)/(S.d) of every face, rounded exactly as the face assembly does
cudaError_t launch_face_c(int32_t n, int32_t F, const int32_t *owner, const int32_t *neighbour, const double *Sf,
                          const double *C, double *c, cudaStream_t s);

// Dictionary of the compact table: dict[2k] = (float)(c_k / rho_w),
// dict[2k+1] = (float)(c_k / rho_a) for geometric class k (densities of the
// class's tank when batched), dict[2 n_cls] = 0, each rounded exactly as the
// face assembly rounds gamma_f off the interface.
struct DictArgs {
    int32_t n_cls;
    const double *ccls;
    const int32_t *ctank;    // batched: tank of each class (else nullptr)
    const TankPhys *tphys;
    double rho_w, rho_a;
    float *dict;
};
cudaError_t launch_dict(const DictArgs &a, cudaStream_t s);
cudaError_t launch_bsums(const double *b, int32_t n, DevParams *prm, cudaStream_t s);

struct CoarseArgs {
    int32_t n, F, n_pad;
    const int32_t *owner, *neighbour, *perm;
    const int8_t *kind;
    const double *gamma;
    int32_t ref;  // internal index of the pinned cell, -1 none
    int32_t max_k, min_size, max_cross;
    const DevParams *prm;
    int32_t *parent, *csize, *cand, *counters;  // counters[0] = candidates, [1] = cross faces
    int32_t *bcount, *boff;  // [ceil(F / 256)] cross faces per face block, and their offsets
    double *epart;           // [kCoarseEParts][kMaxCoarse^2] partial sums of E
    int8_t *comp;  // internal order
    CrossFace *cross;
    Coarse *coarse;
    // batched handles (T > 0): coarse regions are chosen per tank (region ids
    // in comp are tank-local)
    int32_t T;
    const int32_t *coff, *ioff;  // [T+1] caller / internal cell offsets of the tanks
    const DevParams *tprm;       // [T] pinned cell and pin of each tank
    TankCoarse *tco;             // [T]
};
cudaError_t launch_coarse(const CoarseArgs &a, cudaStream_t s, int *launches);

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

// ---- gradient and velocity reconstruction (gfm_gradient.cu) ----------------
struct GradArgs {
    Sell m;
    int32_t n, F;
    const int32_t *iperm;              // internal -> caller (-1 padding)
    const int32_t *owner, *neighbour;  // caller order
    const double *Sf, *C, *V, *xf;     // xf nullable: face centres half-way between cell centres
    const double *lambda, *jump;       // assembled interface fraction and oriented jump
    const double *p;                   // caller order p_d
    const double *phi;                 // face flux for U (nullable when U is)
    double rho_w, rho_a;
    const int32_t *stank;              // batched: tank of each slice (else nullptr)
    const TankPhys *tphys;             // batched: densities per tank
    double *grad, *U;                  // [3][n] caller order, either nullable
};
cudaError_t launch_gradient(const GradArgs &a, cudaStream_t s);

// Explicit non-orthogonal correction: corr_f = rau_f k_f . G_f from the
// cell gradient G [3][n] (caller order), phi_eff = phi - corr and
// sigma = phi_eff + gamma J for the cell sums.
struct NonorthArgs {
    int32_t n, F;
    const int32_t *owner, *neighbour;
    const double *Sf, *C, *xf;  // xf nullable
    const double *rau;          // nullable
    const double *G;
    const double *phi, *gamma, *jump;
    double *corr, *phi_eff, *sigma;
};
cudaError_t launch_nonorth(const NonorthArgs &a, cudaStream_t s);

// ---- isoAdvector advection step (gfm_iso.cu) ------------------------------
struct IsoArgs {
    Sell m;
    int32_t n, F, nvt;
    const int32_t *iperm, *owner, *neighbour;
    const double *alpha, *phi;
    double dt;
    const int32_t *fv_ptr;   // [F+1]
    const double *fv_xyz;    // [3][nvt]
    const double *xf;        // [3][F] triangle apexes
    const int8_t *has_iso;   // [n]
    const double *xS, *nS;   // [3][n]
    const double *UnS;       // [n]
    const double *V;         // [n]
    double *integral;        // [F] nullable
    double *dV;              // [F]
    double *alpha_new;       // [n] nullable
};
cudaError_t launch_iso(const IsoArgs &a, cudaStream_t s);

cudaError_t launch_gather(const double *src_user, const int32_t *iperm, double *dst_internal, int32_t n,
                          int32_t n_pad, cudaStream_t s);

// ---- solver (gfm_solve.cu) ----------------------------------------------
// Batched solve: every CTA works on one tank (cta[b] = {tank, s0, s1, end},
// end = internal index one past the tank's last real cell); tank_cta[t] =
// {first CTA, one past the last}.
struct BatchArgs {
    int32_t T;
    const int4 *cta;
    const int2 *tank_cta;
    const DevParams *tprm;
    gfm_solve_info *infos;  // [T]
    const TankCoarse *tco;  // [T] coarse space of each tank
};
const void *batched_kernel(int max_width, bool streamed = false, bool compact = false);

enum class Mode { FP64 = 0, MIXED = 1 };
const void *solver_kernel(Mode m, int max_width, int threads, bool streamed = false, bool compact = false,
                          bool fused = false);
int solver_max_threads();

}  // namespace gfm
