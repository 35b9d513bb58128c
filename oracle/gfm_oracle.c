/*
 * gfm_oracle.c -- plain, slow, CPU FP64 oracle for the Ghost Fluid Method
 * dynamic-pressure equation of Vukcevic, Roenby, Gatin & Jasak, "A sharp free
 * surface finite volume method applied to gravity wave flows" (Sec. 3.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path and never calls it.
 *
 * Conventions.  n cells, F internal faces; face f has owner[f] < neighbour[f],
 * area vector Sf[k*F+f] pointing owner -> neighbour, cell centres C[k*n+i].
 * Boundary faces are walls (zero flux, zero-gradient p_d) and do not appear.
 * Superscript + is the heavy fluid (water, "wet", rho_w), - the light fluid
 * (air, "dry", rho_a), as in Eq. 4.
 *
 * Readings taken where the paper is silent or inconsistent:
 *  - jump sign: Eq. 7 ([p_d] = -[rho] g.x with [rho] = rho- - rho+, Eq. 4),
 *    i.e. H = p_d- - p_d+ = (rho_w - rho_a) g.x_Gamma.  Eq. 15 prints the
 *    opposite sign; with that sign still water would not stay still.
 *  - alpha == 0.5 exactly counts as wet (the paper leaves it unassigned).
 *  - lambda is measured from the wet cell of an interface face (Eq. 13 with
 *    P = wet cell); non-interface faces use the phase's own density.
 *  - Rhie-Chow 1/a_P factor taken as 1: the predicted flux phi* is an input.
 *  - non-orthogonal correction: implicit part only, c_f = (S.S)/(S.d).
 *  - reference level: OpenFOAM-style pin of one cell (diag doubled, source
 *    increased by diag * value), keeping the matrix symmetric positive definite.
 *
 * Parity is pinned by the CPU tests (still water, symmetry and zero row sums,
 * dense Cholesky, 1D column closed form, literal ghost-value route of
 * Eqs. 17-20, single-phase eigenvectors, translation invariance, finite
 * differences of the adjoint).
 *
 * Floating point: build with -O2 -ffp-contract=off and no fast-math, so every
 * expression below rounds exactly as written, left to right.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KIND_DRY 0        /* both cells dry                 */
#define KIND_WET 1        /* both cells wet                 */
#define KIND_IF_OWNER_WET 2  /* interface face, owner wet   */
#define KIND_IF_OWNER_DRY 3  /* interface face, owner dry   */

/* Planted-mistake switches used only by the tests that prove the pins
 * catch plausible errors.  0 means the faithful oracle. */
#define MUT_NONE 0
#define MUT_JUMP_SIGN_EQ15 1    /* use Eq. 15's printed sign for the jump     */
#define MUT_LAMBDA_FROM_OWNER 2 /* measure lambda from the owner, not wet side */
#define MUT_ARITH_BETA 3        /* arithmetic mean of beta instead of Eq. 18   */
#define MUT_DROP_JUMP 4         /* drop the jump source                        */
#define MUT_SWAP_ALPHA_DERIV 5  /* swap d lambda/d alpha_W and d alpha_D        */
#define MUT_PCG_NO_PRECOND 6    /* fixed-count PCG: drop the Jacobi weights      */
#define MUT_PCG_STALE_RZ 7      /* fixed-count PCG: never update r.z             */
#define MUT_GHOST_SWAP_BETA 8   /* gradient: wet-side ghost weighted by beta+    */
#define MUT_NONORTH_SIGN 9      /* non-orthogonal correction added, not removed  */
#define MUT_ISO_DOWNWIND 10     /* isoAdvector: interface of the downwind cell   */

int gfm_oracle_version(void) { return 3; }

void gfm_oracle_set_threads(int nt)
{
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
#else
    (void)nt;
#endif
}

int gfm_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Per-face interface quantities (Sec. 3.1):
 *   wet_i = alpha_i >= 0.5                      (wet/dry cells, alpha = 0.5 contour)
 *   interface face  iff wet_owner != wet_neighbour
 *   lambda_W = (alpha_W - 0.5)/(alpha_W - alpha_D)  (Eq. 13, P = wet cell W)
 *   x_Gamma = x_W + lambda_W (x_D - x_W)             (Eq. 12)
 *   H = p_d(dry side) - p_d(wet side) = (rho_w - rho_a) g.x_Gamma  (Eq. 7)
 *   face coefficient gamma_f = c_f * beta+ beta- / beta_w
 *                            = c_f / (lambda_W rho_w + (1 - lambda_W) rho_a)
 *     (Eqs. 16-18 and 20 collapsed: the flux from the wet side through the
 *      ghost value of Eq. 20 is gamma_f (p_D - p_W - H)), with
 *   c_f = (S_f.S_f)/(S_f.d_f), d_f = C_neighbour - C_owner.
 *   Oriented jump J_f: flux owner->neighbour is gamma_f (p_nb - p_own - J_f),
 *   so J_f = +H if the owner is wet, -H if it is dry, 0 off the interface.
 * Non-interface faces: lambda = 1 (both wet) or 0 (both dry), which gives the
 * phase's own density exactly.
 * With a Rhie-Chow coefficient per face (rau, the face value of 1/a_P of the
 * momentum equation, Sec. 3; NULL = 1) the face coefficient is
 * gamma_f = (c_f / rho_f) * rau_f: the pressure equation is then
 * div(rau beta grad p_d) = div(phi*), and the jump term scales with it.
 */
int gfm_oracle_faces(int n, int F, const int32_t *owner, const int32_t *neighbour,
                     const double *Sf, const double *C, const double *alpha,
                     double rho_w, double rho_a, const double *g, const double *rau,
                     double *lambda, double *gamma, double *jump, int8_t *kind, int mutate)
{
    for (int f = 0; f < F; ++f) {
        int o = owner[f], nb = neighbour[f];
        if (o < 0 || nb < 0 || o >= n || nb >= n || o >= nb) return -1;
        double ao = alpha[o], an = alpha[nb];
        int wo = ao >= 0.5, wn = an >= 0.5;
        int k;
        double lam;
        int W = o, D = nb;
        if (wo && wn) { k = KIND_WET; lam = 1.0; }
        else if (!wo && !wn) { k = KIND_DRY; lam = 0.0; }
        else {
            if (wo) { k = KIND_IF_OWNER_WET; W = o; D = nb; }
            else { k = KIND_IF_OWNER_DRY; W = nb; D = o; }
            if (mutate == MUT_LAMBDA_FROM_OWNER) { W = o; D = nb; }
            double aW = alpha[W], aD = alpha[D];
            lam = (aW - 0.5) / (aW - aD);
        }
        double Sx = Sf[0 * (size_t)F + f], Sy = Sf[1 * (size_t)F + f], Sz = Sf[2 * (size_t)F + f];
        double dx = C[0 * (size_t)n + nb] - C[0 * (size_t)n + o];
        double dy = C[1 * (size_t)n + nb] - C[1 * (size_t)n + o];
        double dz = C[2 * (size_t)n + nb] - C[2 * (size_t)n + o];
        double c = (Sx * Sx + Sy * Sy + Sz * Sz) / (Sx * dx + Sy * dy + Sz * dz);
        double gam;
        if (mutate == MUT_ARITH_BETA && (k == KIND_IF_OWNER_WET || k == KIND_IF_OWNER_DRY)) {
            gam = c * (lam * (1.0 / rho_w) + (1.0 - lam) * (1.0 / rho_a));
        } else {
            double rf = lam * rho_w + (1.0 - lam) * rho_a;
            gam = c / rf;
        }
        if (rau) gam = gam * rau[f]; /* Rhie-Chow 1/a_P of the face, when given */
        double J = 0.0;
        if (k == KIND_IF_OWNER_WET || k == KIND_IF_OWNER_DRY) {
            double xg0 = C[0 * (size_t)n + W] + lam * (C[0 * (size_t)n + D] - C[0 * (size_t)n + W]);
            double xg1 = C[1 * (size_t)n + W] + lam * (C[1 * (size_t)n + D] - C[1 * (size_t)n + W]);
            double xg2 = C[2 * (size_t)n + W] + lam * (C[2 * (size_t)n + D] - C[2 * (size_t)n + W]);
            double H = (rho_w - rho_a) * ((g[0] * xg0 + g[1] * xg1) + g[2] * xg2);
            if (mutate == MUT_JUMP_SIGN_EQ15) H = -H;
            if (mutate == MUT_DROP_JUMP) H = 0.0;
            J = (k == KIND_IF_OWNER_WET) ? H : -H;
        }
        lambda[f] = lam;
        gamma[f] = gam;
        jump[f] = J;
        kind[f] = (int8_t)k;
    }
    return 0;
}

/*
 * Cell assembly of the discrete continuity equation (Eq. 1 with the GFM
 * Laplacian, symmetric as stated in Sec. 3.1):
 *   for every cell i:  sum_{f in i} s_if phi_f = 0,
 *   phi_f = phi*_f - gamma_f (p_nb - p_own - J_f)   (corrected face flux),
 * which gives A p = b with
 *   A_ii = sum_{f in i} gamma_f,  A_{o,nb} = A_{nb,o} = -gamma_f,
 *   b_i  = - sum_{f in i} s_if (phi*_f + gamma_f J_f),  s = +1 owner, -1 neighbour.
 * Per-cell sums run over faces in ascending face index.  Pin (reference level):
 *   b_r += A_rr * p_ref;  A_rr += A_rr   (skipped when ref_cell < 0).
 * Output is CSR with each row's columns ascending; nnz = n + 2F.
 * diag[] and b[] are also returned on their own.
 */
int gfm_oracle_assemble(int n, int F, const int32_t *owner, const int32_t *neighbour,
                        const double *gamma, const double *jump, const double *phi,
                        int ref_cell, double ref_value,
                        int64_t *rowptr, int32_t *col, double *val, double *diag, double *b)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *pos = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!cnt || !pos) { free(cnt); free(pos); return -2; }
    for (int i = 0; i < n; ++i) { diag[i] = 0.0; b[i] = 0.0; cnt[i + 1] = 1; }
    for (int f = 0; f < F; ++f) {
        int o = owner[f], nb = neighbour[f];
        if (o < 0 || nb < 0 || o >= n || nb >= n || o >= nb) { free(cnt); free(pos); return -1; }
        double sig = phi[f] + gamma[f] * jump[f];
        diag[o] = diag[o] + gamma[f];
        diag[nb] = diag[nb] + gamma[f];
        b[o] = b[o] - sig;
        b[nb] = b[nb] + sig;
        cnt[o + 1] += 1;
        cnt[nb + 1] += 1;
    }
    if (ref_cell >= 0) {
        if (ref_cell >= n) { free(cnt); free(pos); return -1; }
        b[ref_cell] = b[ref_cell] + diag[ref_cell] * ref_value;
        diag[ref_cell] = diag[ref_cell] + diag[ref_cell];
    }
    rowptr[0] = 0;
    for (int i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + cnt[i + 1];
    /* fill every row (off-diagonals by face, then the diagonal), then sort
     * each row by column (insertion sort; rows are short). */
    for (int i = 0; i < n; ++i) pos[i] = rowptr[i];
    for (int f = 0; f < F; ++f) {
        int o = owner[f], nb = neighbour[f];
        col[pos[o]] = nb; val[pos[o]] = -gamma[f]; pos[o]++;
        col[pos[nb]] = o; val[pos[nb]] = -gamma[f]; pos[nb]++;
    }
    for (int i = 0; i < n; ++i) { col[pos[i]] = i; val[pos[i]] = diag[i]; pos[i]++; }
    for (int i = 0; i < n; ++i) {
        for (int64_t a = rowptr[i] + 1; a < rowptr[i + 1]; ++a) {
            int32_t cc = col[a]; double vv = val[a]; int64_t q = a - 1;
            while (q >= rowptr[i] && col[q] > cc) { col[q + 1] = col[q]; val[q + 1] = val[q]; --q; }
            col[q + 1] = cc; val[q + 1] = vv;
        }
    }
    free(cnt); free(pos);
    return 0;
}

/* y = A x for a CSR matrix. */
void gfm_oracle_spmv(int n, const int64_t *rowptr, const int32_t *col, const double *val,
                     const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t a = rowptr[i]; a < rowptr[i + 1]; ++a) s = s + val[a] * x[col[a]];
        y[i] = s;
    }
}

static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/*
 * Jacobi-preconditioned conjugate gradients (the paper names no solver; it
 * reports residual levels only, Sec. 4.1.1).  Textbook PCG on the SPD pinned
 * system, preconditioner M = diag(A), starting from the x passed in.  Stops
 * when the TRUE relative residual ||b - A x||_2 / ||b||_2 <= rtol: the
 * recurrence residual is used to decide when to check, and on a miss the
 * iteration restarts from the true residual.  Returns 0 when converged, 1 when
 * maxit was reached, 2 on breakdown.  iters_out / relres_out report the result.
 * If ref_cell < 0 the system is singular but consistent; CG still converges.
 */
int gfm_oracle_pcg(int n, const int64_t *rowptr, const int32_t *col, const double *val,
                   const double *b, double *x, double rtol, int maxit,
                   int *iters_out, double *relres_out)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double *dinv = (double *)malloc(sizeof(double) * (size_t)n);
    if (!r || !z || !p || !q || !dinv) { free(r); free(z); free(p); free(q); free(dinv); return -2; }
    for (int i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t a = rowptr[i]; a < rowptr[i + 1]; ++a) if (col[a] == i) d = val[a];
        dinv[i] = 1.0 / d;
    }
    double bn = sqrt(dot(n, b, b));
    if (bn == 0.0) bn = 1.0;
    int it = 0, status = 1;
    double rel = 0.0;
    for (int restart = 0; restart < 50 && it < maxit; ++restart) {
        gfm_oracle_spmv(n, rowptr, col, val, x, q);
        for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
        rel = sqrt(dot(n, r, r)) / bn;
        if (rel <= rtol) { status = 0; break; }
        for (int i = 0; i < n; ++i) { z[i] = dinv[i] * r[i]; p[i] = z[i]; }
        double rz = dot(n, r, z);
        int conv = 0;
        while (it < maxit) {
            gfm_oracle_spmv(n, rowptr, col, val, p, q);
            double pq = dot(n, p, q);
            if (!(pq > 0.0)) { status = 2; goto done; }
            double a = rz / pq;
#pragma omp parallel for schedule(static)
            for (int i = 0; i < n; ++i) { x[i] += a * p[i]; r[i] -= a * q[i]; z[i] = dinv[i] * r[i]; }
            ++it;
            double rz2 = dot(n, r, z);
            double rr = sqrt(dot(n, r, r)) / bn;
            if (rr <= rtol) { conv = 1; break; }
            double be = rz2 / rz;
            rz = rz2;
#pragma omp parallel for schedule(static)
            for (int i = 0; i < n; ++i) p[i] = z[i] + be * p[i];
        }
        if (!conv) break;
    }
    gfm_oracle_spmv(n, rowptr, col, val, x, q);
    for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
    rel = sqrt(dot(n, r, r)) / bn;
    if (rel <= rtol) status = 0;
done:
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = rel;
    free(r); free(z); free(p); free(q); free(dinv);
    return status;
}

/*
 * Fixed-count Jacobi-PCG iterations, for timing the oracle on a bounded
 * sample: exactly `iters` iterations of the same textbook recurrence as
 * gfm_oracle_pcg (M = diag(A)) from the x passed in, no convergence test and
 * no restart.  x is overwritten with the k-th iterate; returns ||r_k||_2 of
 * the recurrence residual.  In exact arithmetic the k-th iterate minimises
 * the A-norm of the error over x0 + K_k(M^-1 A, M^-1 r0), the property the
 * CPU tests check it against.  `mutate` plants a mistake for those tests
 * (0 = faithful).
 */
double gfm_oracle_pcg_fixed(int n, const int64_t *rowptr, const int32_t *col, const double *val,
                            const double *b, double *x, int iters, int mutate)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double *dinv = (double *)malloc(sizeof(double) * (size_t)n);
    if (!r || !z || !p || !q || !dinv) { free(r); free(z); free(p); free(q); free(dinv); return -1.0; }
    for (int i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t a = rowptr[i]; a < rowptr[i + 1]; ++a) if (col[a] == i) d = val[a];
        dinv[i] = (mutate == MUT_PCG_NO_PRECOND) ? 1.0 : 1.0 / d;
    }
    gfm_oracle_spmv(n, rowptr, col, val, x, q);
    for (int i = 0; i < n; ++i) { r[i] = b[i] - q[i]; z[i] = dinv[i] * r[i]; p[i] = z[i]; }
    double rz = dot(n, r, z);
    for (int it = 0; it < iters; ++it) {
        gfm_oracle_spmv(n, rowptr, col, val, p, q);
        double pq = dot(n, p, q);
        double a = (pq != 0.0) ? rz / pq : 0.0;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) { x[i] += a * p[i]; r[i] -= a * q[i]; z[i] = dinv[i] * r[i]; }
        double rz2 = dot(n, r, z);
        double be = (rz != 0.0) ? rz2 / rz : 0.0;
        if (mutate != MUT_PCG_STALE_RZ) rz = rz2;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) p[i] = z[i] + be * p[i];
    }
    double rr = sqrt(dot(n, r, r));
    free(r); free(z); free(p); free(q); free(dinv);
    return rr;
}

/*
 * Dense Cholesky solve of the (pinned, SPD) CSR system, textbook
 * column-by-column A = L L^T then two triangular solves.  For small n only
 * (O(n^3) time, n^2 doubles of memory).  Returns 0, or 2 if A is not SPD.
 */
int gfm_oracle_cholesky_solve(int n, const int64_t *rowptr, const int32_t *col, const double *val,
                              const double *b, double *x)
{
    double *L = (double *)calloc((size_t)n * (size_t)n, sizeof(double));
    if (!L) return -2;
    for (int i = 0; i < n; ++i)
        for (int64_t a = rowptr[i]; a < rowptr[i + 1]; ++a) L[(size_t)i * n + col[a]] = val[a];
    for (int j = 0; j < n; ++j) {
        double s = L[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) { free(L); return 2; }
        double d = sqrt(s);
        L[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = L[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / d;
        }
    }
    for (int i = 0; i < n; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * x[k];
        x[i] = t / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = x[i];
        for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * x[k];
        x[i] = t / L[(size_t)i * n + i];
    }
    free(L);
    return 0;
}

/*
 * Corrected face flux (the flux the p_d solution leaves after the GFM
 * gradient is subtracted from the predicted flux; zero in still water):
 *   phi_f = phi*_f - gamma_f (p_nb - p_own - J_f).
 * The discrete continuity equation says sum_f s_if phi_f = 0 in every cell
 * (except the pinned one, which absorbs the solver residual).
 */
void gfm_oracle_corrected_flux(int F, const int32_t *owner, const int32_t *neighbour,
                               const double *gamma, const double *jump, const double *phi,
                               const double *p, double *out)
{
    for (int f = 0; f < F; ++f) {
        int o = owner[f], nb = neighbour[f];
        out[f] = phi[f] - gamma[f] * ((p[nb] - p[o]) - jump[f]);
    }
}

/*
 * Literal ghost-value route of Sec. 3.1, for cross-checking the collapsed
 * coefficient: for every interface face with P = wet cell, N = dry cell,
 *   beta+ = 1/rho_w, beta- = 1/rho_a                         (Eq. 14)
 *   lambda = (alpha_P - 0.5)/(alpha_P - alpha_N)              (Eq. 13)
 *   x_Gamma = x_P + lambda d_f                                (Eq. 12)
 *   H = p_d- - p_d+ = -[rho] g.x_Gamma, [rho] = rho- - rho+   (Eqs. 4, 7)
 *   beta_w = lambda beta- + (1 - lambda) beta+                (Eq. 18)
 *   p+ = (lambda beta-/beta_w) p_N + ((1-lambda) beta+/beta_w) p_P
 *        - (lambda beta-/beta_w) H                            (Eq. 17)
 *   p- = p+ + H                                               (Eq. 15, first line)
 *   ghost p_N+ = p+ + ((1-lambda)/lambda)(p+ - p_P)           (Eq. 19)
 * and three fluxes leaving P towards N, each times c_f = |S|^2/(S.d):
 *   q_plus  = beta+ (p+ - p_P)/lambda          (wet one-sided gradient, Eq. 16)
 *   q_minus = beta- (p_N - p-)/(1 - lambda)     (dry one-sided gradient, Eq. 16)
 *   q_ghost = beta+ (p_N+ - p_P)                 (central difference with the ghost, Eq. 20)
 * Outputs are oriented owner -> neighbour.  Non-interface faces get the plain
 * two-point flux beta c (p_nb - p_own) in all three slots.  Faces with
 * lambda == 0 (alpha_P exactly 0.5) get NaN in q_plus and q_ghost.
 * Also returns the jump residual p- - p+ - H (should be 0 up to rounding) and
 * the flux jump q_minus - q_plus (Eq. 16, should be 0).
 */
void gfm_oracle_ghost_route(int n, int F, const int32_t *owner, const int32_t *neighbour,
                            const double *Sf, const double *C, const double *alpha,
                            double rho_w, double rho_a, const double *g, const double *p,
                            double *q_plus, double *q_minus, double *q_ghost, double *pplus, double *pminus)
{
    const double bp = 1.0 / rho_w, bm = 1.0 / rho_a;
    for (int f = 0; f < F; ++f) {
        int o = owner[f], nb = neighbour[f];
        double Sx = Sf[f], Sy = Sf[(size_t)F + f], Sz = Sf[2 * (size_t)F + f];
        double dx = C[nb] - C[o], dy = C[(size_t)n + nb] - C[(size_t)n + o], dz = C[2 * (size_t)n + nb] - C[2 * (size_t)n + o];
        double c = (Sx * Sx + Sy * Sy + Sz * Sz) / (Sx * dx + Sy * dy + Sz * dz);
        int wo = alpha[o] >= 0.5, wn = alpha[nb] >= 0.5;
        if (wo == wn) {
            double be = wo ? bp : bm;
            double fl = be * c * (p[nb] - p[o]);
            q_plus[f] = fl; q_minus[f] = fl; q_ghost[f] = fl;
            pplus[f] = NAN; pminus[f] = NAN;
            continue;
        }
        int P = wo ? o : nb, N = wo ? nb : o;
        double lam = (alpha[P] - 0.5) / (alpha[P] - alpha[N]);
        double xg[3];
        for (int k = 0; k < 3; ++k) xg[k] = C[(size_t)k * n + P] + lam * (C[(size_t)k * n + N] - C[(size_t)k * n + P]);
        double jump_rho = rho_a - rho_w; /* [rho] = rho- - rho+ */
        double H = -jump_rho * (g[0] * xg[0] + g[1] * xg[1] + g[2] * xg[2]);
        double bw = lam * bm + (1.0 - lam) * bp;
        double pp = (lam * bm / bw) * p[N] + ((1.0 - lam) * bp / bw) * p[P] - (lam * bm / bw) * H;
        double pm = pp + H;
        double qp = bp * (pp - p[P]) / lam * c;
        double qm = bm * (p[N] - pm) / (1.0 - lam) * c;
        double ghost = pp + ((1.0 - lam) / lam) * (pp - p[P]);
        double qg = bp * (ghost - p[P]) * c;
        double sgn = (P == o) ? 1.0 : -1.0;
        q_plus[f] = sgn * qp; q_minus[f] = sgn * qm; q_ghost[f] = sgn * qg;
        pplus[f] = pp; pminus[f] = pm;
    }
}

/*
 * Reverse-mode derivative of L(p) through p = A^{-1} b (pinned system), with
 * mu = A^{-1} dL/dp given (A is symmetric, so the adjoint system is A itself).
 *   dL/db = mu,  dL/dA = -mu p^T.
 * With b_i = -sum s_if (phi*_f + gamma_f J_f) and
 * A = sum_f gamma_f (e_o - e_nb)(e_o - e_nb)^T + pin:
 *   dL/dphi*_f  = -(mu_o - mu_nb)
 *   dL/dgamma_f = -(mu_o - mu_nb)(p_o - p_nb + J_f)
 *   dL/dJ_f     = -gamma_f (mu_o - mu_nb)
 * then through the face quantities (interface faces only; wet/dry flags and
 * the pin magnitude held fixed):
 *   gamma = c/rho_f, rho_f = lambda rho_w + (1-lambda) rho_a  => d gamma/d lambda = -gamma (rho_w-rho_a)/rho_f
 *   J = +-(rho_w - rho_a) g.(x_W + lambda (x_D - x_W))        => dJ/d lambda = +-(rho_w-rho_a) g.(x_D - x_W)
 *   lambda = (a_W - 0.5)/(a_W - a_D)  => d lambda/d a_W = (0.5 - a_D)/(a_W - a_D)^2,
 *                                        d lambda/d a_D = (a_W - 0.5)/(a_W - a_D)^2.
 * dL/dalpha is summed per cell in ascending face order.  dL_dlambda may be NULL.
 */
void gfm_oracle_adjoint_chain(int n, int F, const int32_t *owner, const int32_t *neighbour,
                              const double *C, const double *alpha, const double *lambda,
                              const double *gamma, const double *jump, const int8_t *kind,
                              double rho_w, double rho_a, const double *g,
                              const double *p, const double *mu,
                              double *dL_dphi, double *dL_dalpha, double *dL_dlambda, int mutate)
{
    for (int i = 0; i < n; ++i) dL_dalpha[i] = 0.0;
    for (int f = 0; f < F; ++f) {
        int o = owner[f], nb = neighbour[f];
        double dmu = mu[o] - mu[nb];
        dL_dphi[f] = -dmu;
        double dlam = 0.0;
        if (kind[f] == KIND_IF_OWNER_WET || kind[f] == KIND_IF_OWNER_DRY) {
            int W = (kind[f] == KIND_IF_OWNER_WET) ? o : nb;
            int D = (kind[f] == KIND_IF_OWNER_WET) ? nb : o;
            double lam = lambda[f];
            double rf = lam * rho_w + (1.0 - lam) * rho_a;
            double dgam_dlam = -gamma[f] * (rho_w - rho_a) / rf;
            double gd = 0.0;
            for (int k = 0; k < 3; ++k) gd += g[k] * (C[(size_t)k * n + D] - C[(size_t)k * n + W]);
            double dH_dlam = (rho_w - rho_a) * gd;
            double dJ_dlam = (kind[f] == KIND_IF_OWNER_WET) ? dH_dlam : -dH_dlam;
            double dL_dgam = -dmu * ((p[o] - p[nb]) + jump[f]);
            double dL_dJ = -gamma[f] * dmu;
            dlam = dL_dgam * dgam_dlam + dL_dJ * dJ_dlam;
            double aW = alpha[W], aD = alpha[D];
            double den = (aW - aD) * (aW - aD);
            double dW = (0.5 - aD) / den, dD = (aW - 0.5) / den;
            if (mutate == MUT_SWAP_ALPHA_DERIV) { double t = dW; dW = dD; dD = t; }
            dL_dalpha[W] += dlam * dW;
            dL_dalpha[D] += dlam * dD;
        }
        if (dL_dlambda) dL_dlambda[f] = dlam;
    }
}

/*
 * Dynamic-pressure gradient of the momentum equation with the ghost values
 * of Sec. 3.1 (Eq. 2's pressure term (1/rho) grad p_d, Gauss theorem,
 * cell-centre-to-face interpolation corrected at the interface).
 * For each internal face f between cells o and nb, each side P sees the
 * other cell N through a face value
 *   pf(P) = w_P p_P + (1 - w_P) pN~,   w_P = S.(x_N - x_f) / S.(x_N - x_P)
 * (linear interpolation weight from the face centre x_f; the midpoint of the
 * two cell centres when xf is NULL), where pN~ = p_N off the interface and,
 * on an interface face (W wet, D dry, lambda from the wet cell, Eq. 13;
 * x_Gamma by Eq. 12; H = p_d- - p_d+ = (rho_w - rho_a) g.x_Gamma, Eq. 7;
 * beta+ = 1/rho_w, beta- = 1/rho_a, Eq. 14; beta_w by Eq. 18):
 *   seen from W:  pD~ = (beta-/beta_w) p_D + (1 - beta-/beta_w) p_W - (beta-/beta_w) H     (Eq. 20)
 *   seen from D:  pW~ = (beta+/beta_w) p_W + (1 - beta+/beta_w) p_D + (beta+/beta_w) H     (the
 *                 analogous extrapolation into the light fluid: the same jump
 *                 conditions, Eqs. 15-16, solved for p_d- and carried on to W)
 * Walls carry zero-gradient p_d, so their face value is p_P and, the cell
 * being closed, the Gauss sum reduces to the internal faces in difference
 * form:
 *   grad_P = beta_P / V_P * sum_f (pf(P) - p_P) S_Pf,   S_Pf = +S_f (P owner), -S_f (P neighbour),
 * with beta_P = 1/rho of P's own phase (wet: alpha >= 0.5).  Per-cell sums
 * run in ascending face order.  grad is [3][n].  `mutate` plants a mistake
 * for the tests (0 = faithful).
 */
void gfm_oracle_gradient(int n, int F, const int32_t *owner, const int32_t *neighbour,
                         const double *Sf, const double *C, const double *V, const double *xf,
                         const double *alpha, double rho_w, double rho_a, const double *g,
                         const double *p, double *grad, int mutate)
{
    const double bp = 1.0 / rho_w, bm = 1.0 / rho_a;
    for (size_t k = 0; k < 3 * (size_t)n; ++k) grad[k] = 0.0;
    for (int f = 0; f < F; ++f) {
        int o = owner[f], nb = neighbour[f];
        double S[3], x[3];
        for (int k = 0; k < 3; ++k) {
            S[k] = Sf[(size_t)k * F + f];
            x[k] = xf ? xf[(size_t)k * F + f] : 0.5 * (C[(size_t)k * n + o] + C[(size_t)k * n + nb]);
        }
        /* weights: w_o = S.(x_nb - x_f)/S.d, w_nb = S.(x_f - x_o)/S.d */
        double sd = 0.0, snf = 0.0, sfo = 0.0;
        for (int k = 0; k < 3; ++k) {
            double xo = C[(size_t)k * n + o], xn = C[(size_t)k * n + nb];
            sd += S[k] * (xn - xo);
            snf += S[k] * (xn - x[k]);
            sfo += S[k] * (x[k] - xo);
        }
        double w_o = snf / sd, w_nb = sfo / sd;
        int wo = alpha[o] >= 0.5, wn = alpha[nb] >= 0.5;
        double ghost_for_o = p[nb], ghost_for_nb = p[o];
        if (wo != wn) {
            int W = wo ? o : nb, D = wo ? nb : o;
            double lam = (alpha[W] - 0.5) / (alpha[W] - alpha[D]);
            double xg[3];
            for (int k = 0; k < 3; ++k)
                xg[k] = C[(size_t)k * n + W] + lam * (C[(size_t)k * n + D] - C[(size_t)k * n + W]);
            double H = -(rho_a - rho_w) * (g[0] * xg[0] + g[1] * xg[1] + g[2] * xg[2]);
            if (mutate == MUT_JUMP_SIGN_EQ15) H = -H;
            if (mutate == MUT_DROP_JUMP) H = 0.0;
            double bw = lam * bm + (1.0 - lam) * bp;
            double rW = (mutate == MUT_GHOST_SWAP_BETA) ? bp / bw : bm / bw;
            double gD = rW * p[D] + (1.0 - rW) * p[W] - rW * H; /* D's value seen from W */
            double gW = (bp / bw) * p[W] + (1.0 - bp / bw) * p[D] + (bp / bw) * H; /* W's value seen from D */
            if (W == o) { ghost_for_o = gD; ghost_for_nb = gW; }
            else { ghost_for_o = gW; ghost_for_nb = gD; }
        }
        double pf_o = w_o * p[o] + (1.0 - w_o) * ghost_for_o;
        double pf_nb = w_nb * p[nb] + (1.0 - w_nb) * ghost_for_nb;
        for (int k = 0; k < 3; ++k) {
            grad[(size_t)k * n + o] += (pf_o - p[o]) * S[k];
            grad[(size_t)k * n + nb] -= (pf_nb - p[nb]) * S[k];
        }
    }
    for (int i = 0; i < n; ++i) {
        double be = (alpha[i] >= 0.5) ? bp : bm;
        for (int k = 0; k < 3; ++k) grad[(size_t)k * n + i] = be * grad[(size_t)k * n + i] / V[i];
    }
}

/*
 * Cell velocity from face fluxes (the flux/velocity reconstruction that
 * follows the pressure solve): for a closed cell, sum_f (u.S_f)(x_f - x_P)
 * = V_P u for any uniform u, so
 *   U_P = 1/V_P * sum_f phi_Pf (x_f - x_P),   phi_Pf = +phi_f (P owner), -phi_f (P neighbour),
 * over internal faces; wall faces carry no flux.  Face centres as in
 * gfm_oracle_gradient (midpoints when xf is NULL).  U is [3][n].
 */
void gfm_oracle_reconstruct(int n, int F, const int32_t *owner, const int32_t *neighbour,
                            const double *C, const double *V, const double *xf, const double *phi, double *U)
{
    for (size_t k = 0; k < 3 * (size_t)n; ++k) U[k] = 0.0;
    for (int f = 0; f < F; ++f) {
        int o = owner[f], nb = neighbour[f];
        for (int k = 0; k < 3; ++k) {
            double x = xf ? xf[(size_t)k * F + f] : 0.5 * (C[(size_t)k * n + o] + C[(size_t)k * n + nb]);
            U[(size_t)k * n + o] += phi[f] * (x - C[(size_t)k * n + o]);
            U[(size_t)k * n + nb] -= phi[f] * (x - C[(size_t)k * n + nb]);
        }
    }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) U[(size_t)k * n + i] /= V[i];
}

/*
 * Explicit non-orthogonal correction of the face flux (Sec. 3: the
 * over-relaxed approach, treated explicitly).  The area vector splits into
 * a part along the centre-to-centre vector d and a remainder:
 *   S_f = Delta_f + k_f,   Delta_f = (S_f.S_f)/(S_f.d_f) d_f  (over-relaxed),
 * the Delta part being the implicit two-point term c_f (p_nb - p_own) of the
 * pressure equation.  The k part uses the gradient of the last p_d:
 *   corr_f = rau_f k_f . G_f,   G_f = w_o G_own + (1 - w_o) G_nb,
 * G = (1/rho) grad p_d of gfm_oracle_gradient (continuous across the
 * interface by Eq. 8, so it is interpolated as it stands), w_o the linear
 * weight from the face centre.  The face flux becomes
 *   phi_f = phi*_f - corr_f - gamma_f (p_nb - p_own - J_f),
 * i.e. the assembly takes phi* - corr in place of phi*.  rau NULL = 1;
 * xf NULL = midpoints.  corr is [F].  `mutate` plants a mistake for the
 * tests (0 = faithful).
 */
void gfm_oracle_nonorth(int n, int F, const int32_t *owner, const int32_t *neighbour,
                        const double *Sf, const double *C, const double *V, const double *xf,
                        const double *alpha, double rho_w, double rho_a, const double *g,
                        const double *rau, const double *p, double *corr, int mutate)
{
    double *G = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!G) return;
    gfm_oracle_gradient(n, F, owner, neighbour, Sf, C, V, xf, alpha, rho_w, rho_a, g, p, G, 0);
    for (int f = 0; f < F; ++f) {
        int o = owner[f], nb = neighbour[f];
        double S[3], d[3], x[3];
        for (int k = 0; k < 3; ++k) {
            S[k] = Sf[(size_t)k * F + f];
            d[k] = C[(size_t)k * n + nb] - C[(size_t)k * n + o];
            x[k] = xf ? xf[(size_t)k * F + f] : 0.5 * (C[(size_t)k * n + o] + C[(size_t)k * n + nb]);
        }
        double ss = S[0] * S[0] + S[1] * S[1] + S[2] * S[2];
        double sd = S[0] * d[0] + S[1] * d[1] + S[2] * d[2];
        double snf = 0.0;
        for (int k = 0; k < 3; ++k) snf += S[k] * (C[(size_t)k * n + nb] - x[k]);
        double w_o = snf / sd;
        double kg = 0.0;
        for (int k = 0; k < 3; ++k) {
            double kf = S[k] - (ss / sd) * d[k];
            double Gf = w_o * G[(size_t)k * n + o] + (1.0 - w_o) * G[(size_t)k * n + nb];
            kg += kf * Gf;
        }
        corr[f] = (rau ? rau[f] : 1.0) * kg;
        if (mutate == MUT_NONORTH_SIGN) corr[f] = -corr[f];
    }
    free(G);
}

/*
 * isoAdvector advection step (Sec. 3.2), face fluxes by their plain
 * definition.  Over the time step [0, dt] the heavy-fluid volume through face
 * f is dV_f = phi_f * I_f with I_f = int_0^dt alpha_f+(tau) dtau (Eq. dV),
 * alpha_f+ the submerged fraction of the face area (Eq. alphaf).  The face
 * surface is the union of the triangles (apex x_f, v_k, v_k+1) over its N
 * edges.  In the upwind cell U (owner if phi_f >= 0, else neighbour) the
 * interface is the plane through x_S[U] with unit normal n_S[U] (pointing
 * away from the heavy fluid) moving along n_S at speed Un_S[U], so a point x
 * is in heavy fluid at time tau iff (x - x_S).n_S < Un_S tau.  If U has no
 * isoface (has_iso[U] == 0) the face carries alpha_U throughout.
 * The submerged area of each triangle at time tau is found by clipping the
 * triangle with that half-space (Sutherland-Hodgman) and taking the area of
 * the clipped polygon; between consecutive arrival times of the triangle's
 * vertices it is a quadratic in tau, so two-point Gauss-Legendre on each
 * such sub-interval of [0, dt] integrates it exactly.
 * fv_ptr [F+1], fv_xyz [3][nvt] (vertices of each face in order round it),
 * xf [3][F] apexes; integral [F] = I_f, dV [F] = phi_f I_f.  `mutate` plants
 * a mistake for the tests (0 = faithful).
 */
static double tri_area3(const double *a, const double *b, const double *c)
{
    double u[3], v[3];
    for (int k = 0; k < 3; ++k) { u[k] = b[k] - a[k]; v[k] = c[k] - a[k]; }
    double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    return 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

/* area of triangle (a, b, c) where (x - xS).n < level */
static double clipped_area(const double *a, const double *b, const double *c, const double *xS, const double *nS,
                           double level)
{
    const double *P[3] = {a, b, c};
    double out[4][3];
    int m = 0;
    for (int i = 0; i < 3; ++i) {
        const double *p = P[i], *q = P[(i + 1) % 3];
        double sp = 0.0, sq = 0.0;
        for (int k = 0; k < 3; ++k) { sp += (p[k] - xS[k]) * nS[k]; sq += (q[k] - xS[k]) * nS[k]; }
        sp -= level;
        sq -= level;
        int pin = sp < 0.0, qin = sq < 0.0;
        if (pin) { for (int k = 0; k < 3; ++k) out[m][k] = p[k]; ++m; }
        if (pin != qin) {
            double t = sp / (sp - sq);
            for (int k = 0; k < 3; ++k) out[m][k] = p[k] + t * (q[k] - p[k]);
            ++m;
        }
    }
    double A = 0.0;
    for (int i = 1; i + 1 < m; ++i) A += tri_area3(out[0], out[i], out[i + 1]);
    return A;
}

static void sort3(double *t)
{
    double a;
    if (t[0] > t[1]) { a = t[0]; t[0] = t[1]; t[1] = a; }
    if (t[1] > t[2]) { a = t[1]; t[1] = t[2]; t[2] = a; }
    if (t[0] > t[1]) { a = t[0]; t[0] = t[1]; t[1] = a; }
}

void gfm_oracle_iso_flux(int n, int F, const int32_t *owner, const int32_t *neighbour, const double *alpha,
                         const double *phi, double dt, const int32_t *fv_ptr, const double *fv_xyz, int nvt,
                         const double *xf, const int8_t *has_iso, const double *xS, const double *nS,
                         const double *UnS, double *integral, double *dV, int mutate)
{
    const double gx = 0.5773502691896257645; /* 1/sqrt(3): two-point Gauss-Legendre nodes on [-1, 1] */
    for (int f = 0; f < F; ++f) {
        int U = phi[f] >= 0.0 ? owner[f] : neighbour[f];
        if (mutate == MUT_ISO_DOWNWIND) U = phi[f] >= 0.0 ? neighbour[f] : owner[f];
        double I;
        if (!has_iso[U]) {
            I = alpha[U] * dt;
        } else {
            double xs[3], ns[3], apex[3];
            for (int k = 0; k < 3; ++k) {
                xs[k] = xS[(size_t)k * n + U];
                ns[k] = nS[(size_t)k * n + U];
                apex[k] = xf[(size_t)k * F + f];
            }
            double un = UnS[U];
            double Atot = 0.0, acc = 0.0;
            int v0 = fv_ptr[f], nv = fv_ptr[f + 1] - fv_ptr[f];
            for (int e = 0; e < nv; ++e) {
                double va[3], vb[3];
                for (int k = 0; k < 3; ++k) {
                    va[k] = fv_xyz[(size_t)k * nvt + v0 + e];
                    vb[k] = fv_xyz[(size_t)k * nvt + v0 + (e + 1) % nv];
                }
                double At = tri_area3(apex, va, vb);
                Atot += At;
                if (At == 0.0) continue;
                if (un == 0.0) {
                    acc += clipped_area(apex, va, vb, xs, ns, 0.0) * dt;
                    continue;
                }
                /* breakpoints: arrival times of the three vertices, clipped to [0, dt] */
                double t[3];
                const double *V3[3] = {apex, va, vb};
                for (int i = 0; i < 3; ++i) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += (V3[i][k] - xs[k]) * ns[k];
                    t[i] = s / un;
                }
                sort3(t);
                double br[5] = {0.0, t[0], t[1], t[2], dt};
                for (int i = 1; i < 4; ++i) br[i] = br[i] < 0.0 ? 0.0 : (br[i] > dt ? dt : br[i]);
                for (int i = 0; i < 4; ++i) {
                    double lo = br[i], hi = br[i + 1];
                    if (!(hi > lo)) continue;
                    double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
                    double a1 = clipped_area(apex, va, vb, xs, ns, un * (mid - half * gx));
                    double a2 = clipped_area(apex, va, vb, xs, ns, un * (mid + half * gx));
                    acc += half * (a1 + a2);
                }
            }
            I = Atot > 0.0 ? acc / Atot : 0.0;
        }
        integral[f] = I;
        dV[f] = phi[f] * I;
    }
}

/*
 * Volume-fraction update of the advection step (Sec. 3.2):
 *   alpha_P(t + dt) = alpha_P(t) - 1/V_P sum_f s_Pf dV_f,
 * s = +1 where P owns f (flux leaves P), -1 where it is the neighbour; sums
 * in ascending face order.
 */
void gfm_oracle_iso_advect(int n, int F, const int32_t *owner, const int32_t *neighbour, const double *V,
                           const double *alpha, const double *dV, double *alpha_new)
{
    double *acc = (double *)calloc((size_t)n, sizeof(double));
    if (!acc) return;
    for (int f = 0; f < F; ++f) {
        acc[owner[f]] += dV[f];
        acc[neighbour[f]] -= dV[f];
    }
    for (int i = 0; i < n; ++i) alpha_new[i] = alpha[i] - acc[i] / V[i];
    free(acc);
}
