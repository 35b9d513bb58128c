"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
balanced-force still-water state (Eqs. 3, 7, 8), the symmetry stated in
Sec. 3.1, a dense direct solve, a 1D closed form derived from the jump
conditions (Eqs. 15-16) as two half-cell resistances in series, the literal
ghost-value route (Eqs. 17-20), exact eigenpairs of the single-phase
Laplacian, translation invariance of the physical pressure (Eq. 3), and
finite differences of the adjoint.  The planted-mistake tests at the end show
that each plausible error in the oracle makes at least one pin fail.
"""
import math

import numpy as np
import pytest

import cases
import oracle


def _still(nx=16, ny=8, nz=1, level=0.4475, permute_seed=None):
    c = cases.still_water_case(nx=nx, ny=ny, nz=nz, level=level)
    if permute_seed is not None:
        mesh = dict(n=c.n, F=c.F, owner=c.owner, neighbour=c.neighbour, Sf=c.Sf, C=c.C, V=c.V, xf=c.xf,
                    dims=c.dims)
        perm = np.random.default_rng(permute_seed).permutation(c.n)
        pm = cases.permute_mesh(mesh, perm, face_fields=(c.phi,))
        alpha = np.empty_like(c.alpha)
        alpha[perm] = c.alpha
        c = cases.Case(name=c.name + "_perm", n=c.n, F=c.F, owner=pm["owner"], neighbour=pm["neighbour"],
                       Sf=pm["Sf"], C=pm["C"], V=pm["V"], xf=pm["xf"], alpha=alpha, phi=pm["fields"][0],
                       ref_cell=int(perm[c.ref_cell]), dims=c.dims)
    return c


# --------------------------------------------------------------------------
# case generator sanity (the inputs both sides read)
# --------------------------------------------------------------------------

def test_case_generator_volume_closed_form():
    """sum(alpha V) equals the exact water volume under eta (Eq. 10)."""
    c = cases.make_case(1)
    dz = 2.0 / 64
    # int_0^2 (0.5 + 0.02 cos 2 pi x) dx = 1.0 exactly
    assert abs(np.sum(c.alpha * c.V) / dz - 1.0) < 1e-13
    assert c.n == 2048 and c.F == 63 * 32 + 64 * 31
    assert np.all(c.owner < c.neighbour)
    # area vectors point owner -> neighbour
    d = c.C[:, c.neighbour] - c.C[:, c.owner]
    assert np.all(np.einsum("kf,kf->f", c.Sf, d) > 0)


def test_case_generator_stokes_volume():
    """Over whole wavelengths the cos terms integrate to zero: volume = d * L."""
    c = cases._wave_tank(256, 64, 16.0, 4.0, 2.0, 0.1, 4, 5, "t", 1e-10, "mixed")
    dz = 16.0 / 256
    assert abs(np.sum(c.alpha * c.V) / dz - 32.0) < 1e-11


def test_permuted_mesh_is_consistent():
    c = cases.box_case(12, 6, 1, permute=True)
    assert np.all(c.owner < c.neighbour)
    order = np.lexsort((c.neighbour, c.owner))
    assert np.array_equal(order, np.arange(c.F))
    d = c.C[:, c.neighbour] - c.C[:, c.owner]
    assert np.all(np.einsum("kf,kf->f", c.Sf, d) > 0)


# --------------------------------------------------------------------------
# pin 1: still water -- balanced force, exact hydrostatics across the jump
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nz,permute", [(1, None), (1, 3), (3, None)])
def test_still_water_is_still_and_hydrostatic(nz, permute):
    c = _still(nz=nz, permute_seed=permute)
    p, fc, sy, info = oracle.solve(c, direct=True)
    q = oracle.corrected_flux(c, fc, p)
    scale = np.max(np.abs(fc.gamma * fc.jump))
    # corrected flux vanishes everywhere (the balanced force stated after Eq. 20, Sec. 3.1)
    assert np.max(np.abs(q)) <= 1e-12 * scale
    wet = c.alpha >= 0.5
    Kw, Ka = p[wet], p[~wet]
    # p_d is constant in each phase
    assert np.ptp(Kw) <= 1e-10 * np.abs(Kw).max()
    assert np.ptp(Ka) <= 1e-10 * max(np.abs(Ka).max(), 1.0)
    # physical pressure p = p_d + rho g.x (Eq. 3) is continuous at some height
    # between the wet and dry cell centres: K_w + rho_w g y = K_a + rho_a g y
    gy = c.g[1]
    y_gamma = (Ka.mean() - Kw.mean()) / ((c.rho_w - c.rho_a) * gy)
    ifc = fc.kind >= 2
    yW = np.where(wet[c.owner[ifc]], c.C[1, c.owner[ifc]], c.C[1, c.neighbour[ifc]])
    yD = np.where(wet[c.owner[ifc]], c.C[1, c.neighbour[ifc]], c.C[1, c.owner[ifc]])
    assert np.all((yW < y_gamma) & (y_gamma < yD))
    # and it sits where alpha = 0.5 is crossed by linear interpolation
    # between the two cell centres (Eqs. 12-13)
    aW = np.max(c.alpha[wet & (c.alpha < 1)])
    dy = 1.0 / 8
    y_expect = yW[0] + (aW - 0.5) / aW * dy
    assert abs(y_gamma - y_expect) < 1e-12
    # hydrostatic physical pressure in water: p = K_w - rho_w |g| y, linear in y
    pw = p[wet] + c.rho_w * gy * c.C[1, wet]
    slope = np.polyfit(c.C[1, wet], pw, 1)[0]
    assert abs(slope - c.rho_w * gy) < 1e-8 * c.rho_w * abs(gy)


# --------------------------------------------------------------------------
# pin 2: symmetry and zero row sums (Sec. 3.1: symmetric Laplacian)
# --------------------------------------------------------------------------

def test_symmetric_zero_row_sum_before_pin():
    c = cases.box_case(16, 8, 1, permute=True)
    fc = oracle.faces(c)
    sy = oracle.assemble(c, fc, ref_cell=-1)
    A = sy.dense()
    assert np.array_equal(A, A.T)
    rows = A.sum(axis=1)
    # diag is the sum of the face coefficients, so row sums vanish up to the
    # rounding of that sum
    assert np.max(np.abs(rows)) <= 8 * np.finfo(float).eps * np.max(np.abs(sy.diag))
    # jump terms only in b: total source telescopes to zero
    assert abs(sy.b.sum()) <= 1e-12 * np.abs(sy.b).sum()
    # pinned: still symmetric, SPD
    sp = oracle.assemble(c, fc)
    Ap = sp.dense()
    assert np.array_equal(Ap, Ap.T)
    assert np.linalg.eigvalsh(Ap).min() > 0
    r = c.ref_cell
    assert Ap[r, r] == 2 * A[r, r]


# --------------------------------------------------------------------------
# pin 3: dense direct solve
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mk", [lambda: cases.make_case(1), lambda: cases.box_case(16, 8, 1),
                                lambda: cases.box_case(8, 4, 1, permute=True)])
def test_pcg_matches_dense_cholesky(mk):
    c = mk()
    fc = oracle.faces(c)
    sy = oracle.assemble(c, fc)
    xd = oracle.cholesky_solve(sy)
    x, it, rel, st = oracle.pcg(sy, rtol=1e-13)
    assert st == 0 and rel <= 1e-13
    assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)
    # and numpy's LAPACK agrees with the textbook Cholesky
    xn = np.linalg.solve(sy.dense(), sy.b)
    assert np.linalg.norm(xn - xd) <= 1e-11 * np.linalg.norm(xd)


# --------------------------------------------------------------------------
# pin 4: 1D column closed form
# --------------------------------------------------------------------------

@pytest.mark.parametrize("level,permute", [(0.43, False), (0.4999, False), (0.43, True)])
def test_column_closed_form(level, permute):
    """1 x N column between walls: continuity forces every corrected flux to
    zero, so each face carries exactly phi*_f.  Across a face the pressure
    drop follows from the one-sided gradients of Eq. 16 and the jump of
    Eq. 15/7: two half-cell resistances in series,
        p_D - p_W = H + phi* |d| (lambda rho_w + (1 - lambda) rho_a) / |S|
    (flux W -> D), and p_N - p_P = phi* |d| rho / |S| in one phase."""
    c = cases.column_case(ny=10, level=level)
    if permute:
        mesh = dict(n=c.n, F=c.F, owner=c.owner, neighbour=c.neighbour, Sf=c.Sf, C=c.C, V=c.V, xf=c.xf,
                    dims=c.dims)
        perm = np.random.default_rng(5).permutation(c.n)
        pm = cases.permute_mesh(mesh, perm, face_fields=(c.phi,))
        alpha = np.empty_like(c.alpha)
        alpha[perm] = c.alpha
        c = cases.Case(name="colp", n=c.n, F=c.F, owner=pm["owner"], neighbour=pm["neighbour"], Sf=pm["Sf"],
                       C=pm["C"], V=pm["V"], xf=pm["xf"], alpha=alpha, phi=pm["fields"][0],
                       ref_cell=int(perm[c.ref_cell]), dims=c.dims)
    p, fc, sy, info = oracle.solve(c, direct=True)
    # walk the column bottom-up in geometric order
    order = np.argsort(c.C[1])
    g = abs(c.g[1])
    pe = np.zeros(c.n)
    pe[order[-1]] = 0.0  # pinned top cell
    face_of = {}
    for f in range(c.F):
        face_of[(c.owner[f], c.neighbour[f])] = f
        face_of[(c.neighbour[f], c.owner[f])] = f
    for k in range(c.n - 2, -1, -1):
        lo, hi = order[k], order[k + 1]
        f = face_of[(lo, hi)]
        sgn = 1.0 if c.owner[f] == lo else -1.0
        flux_up = sgn * c.phi[f]  # predicted flux lo -> hi
        S = np.linalg.norm(c.Sf[:, f])
        d = c.C[1, hi] - c.C[1, lo]
        wl, wh = c.alpha[lo] >= 0.5, c.alpha[hi] >= 0.5
        if wl and wh:
            drop = flux_up * d * c.rho_w / S
        elif not wl and not wh:
            drop = flux_up * d * c.rho_a / S
        else:
            assert wl and not wh
            lam = (c.alpha[lo] - 0.5) / (c.alpha[lo] - c.alpha[hi])
            yg = c.C[1, lo] + lam * d
            # pressure continuity p+ = p- with p = p_d + rho g.x gives the jump
            H = (c.rho_w - c.rho_a) * (-g) * yg
            drop = H + flux_up * d * (lam * c.rho_w + (1 - lam) * c.rho_a) / S
        pe[lo] = pe[hi] - drop
    assert np.max(np.abs(p - pe)) <= 1e-11 * np.max(np.abs(pe))


# --------------------------------------------------------------------------
# pin 5: literal ghost-value route (Eqs. 12-20) == collapsed coefficient
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mk", [lambda: cases.make_case(1), lambda: cases.box_case(10, 8, 3, permute=True,
                                                                                     alpha_noise=0.2)])
def test_ghost_route_equals_collapsed_flux(mk):
    c = mk()
    fc = oracle.faces(c)
    rng = np.random.default_rng(9)
    p = rng.normal(size=c.n) * 1e3  # any pressure field: this is an identity
    qp, qm, qg, pplus, pminus = oracle.ghost_route(c, p)
    flux = fc.gamma * ((p[c.neighbour] - p[c.owner]) - fc.jump)
    ok = np.isfinite(qp)
    scale = np.abs(flux).max()
    for q in (qp, qm, qg):
        assert np.max(np.abs(q[ok] - flux[ok])) <= 1e-9 * scale
    ifc = fc.kind >= 2
    assert ifc.sum() > 0
    # flux continuity [beta grad p_d] = 0 (Eq. 16 = discrete Eq. 8)
    assert np.max(np.abs(qm[ifc & ok] - qp[ifc & ok])) <= 1e-9 * scale
    # jump: p- - p+ = H with H = -[rho] g.x_Gamma (Eq. 7); compare to J
    H = np.where(fc.kind == 2, fc.jump, -fc.jump)
    assert np.max(np.abs((pminus - pplus)[ifc] - H[ifc])) <= 1e-9 * np.abs(H[ifc]).max()


# --------------------------------------------------------------------------
# pin 6: single phase -> standard Neumann Laplacian with known eigenpairs
# --------------------------------------------------------------------------

def test_single_phase_eigenpairs():
    nx, ny = 12, 8
    c = cases.box_case(nx, ny, 1)
    c.alpha = np.ones(c.n)  # all water
    fc = oracle.faces(c)
    assert np.all(fc.jump == 0)
    sy = oracle.assemble(c, fc, ref_cell=-1)
    dx, dy, dz = 2.0 / nx, 1.0 / ny, 2.0 / nx
    cx, cy = dy * dz / dx, dx * dz / dy
    i = np.arange(c.n) % nx
    j = np.arange(c.n) // nx
    for k, l in [(0, 1), (1, 0), (3, 2), (5, 7), (11, 7)]:
        v = np.cos(math.pi * k * (i + 0.5) / nx) * np.cos(math.pi * l * (j + 0.5) / ny)
        lam = (cx * 4 * math.sin(math.pi * k / (2 * nx)) ** 2 + cy * 4 * math.sin(math.pi * l / (2 * ny)) ** 2) / c.rho_w
        Av = oracle.spmv(sy, v)
        assert np.max(np.abs(Av - lam * v)) <= 1e-13 * max(lam, 1e-300) * 10 + 1e-18


# --------------------------------------------------------------------------
# pin 7: translation invariance of the physical pressure (Eq. 3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shift", [(0.3, -0.7, 0.0), (1e4, 1e4, 0.0)])
def test_translation_invariance(shift):
    """Moving the whole problem by c leaves the physical pressure unchanged up
    to a constant, so p_d changes by -rho_phase g.c + K."""
    c = cases.box_case(16, 8, 1)
    p0, fc0, _, _ = oracle.solve(c, direct=True)
    sh = np.asarray(shift)[:, None]
    p1, fc1, _, _ = oracle.solve(c, direct=True, C=c.C + sh)
    wet = c.alpha >= 0.5
    rho = np.where(wet, c.rho_w, c.rho_a)
    gc = float(np.dot(c.g, shift))
    pred = p0 - rho * gc
    pred += p1[c.ref_cell] - pred[c.ref_cell]
    assert np.max(np.abs(p1 - pred)) <= 1e-9 * np.max(np.abs(p1)) + 1e-12 * abs(gc) * c.rho_w


# --------------------------------------------------------------------------
# pin 8: adjoint vs central finite differences
# --------------------------------------------------------------------------

def _band_loss_grad(c):
    band = (np.abs(c.C[0] - 1.0) < 0.3) & (np.abs(c.C[1] - 0.5) < 0.15)
    return np.where(band, c.V, 0.0)


def test_adjoint_matches_central_fd():
    c = cases.box_case(16, 8, 1, alpha_noise=0.05, seed=21)
    w = _band_loss_grad(c)
    dphi, dalpha, mu, p = oracle.adjoint(c, w, direct=True)

    def L(alpha=None, phi=None):
        pp, _, _, _ = oracle.solve(c, direct=True, alpha=alpha, phi=phi)
        return float(np.dot(w, pp))

    rng = np.random.default_rng(3)
    eps = 1e-6
    # phi* enters b affinely, so a central difference is exact for any step;
    # the step is taken at the size of phi* itself so that the difference of L
    # stands far above the rounding of the two solves.
    step_phi = float(np.abs(c.phi).max())
    for f in rng.choice(c.F, 16, replace=False):
        e = np.zeros(c.F)
        e[f] = step_phi
        fd = (L(phi=c.phi + e) - L(phi=c.phi - e)) / (2 * e[f])
        assert abs(fd - dphi[f]) <= 1e-5 * max(abs(dphi[f]), 1e-3 * np.abs(dphi).max())
    fc = oracle.faces(c)
    ifc = np.nonzero(fc.kind >= 2)[0]
    cand = np.unique(np.concatenate([c.owner[ifc], c.neighbour[ifc]]))
    cand = cand[np.abs(c.alpha[cand] - 0.5) > 1e-3]
    for i in rng.choice(cand, min(16, cand.size), replace=False):
        e = np.zeros(c.n)
        e[i] = eps
        fd = (L(alpha=c.alpha + e) - L(alpha=c.alpha - e)) / (2 * eps)
        assert abs(fd - dalpha[i]) <= 1e-5 * max(abs(dalpha[i]), 1e-2 * np.abs(dalpha).max())


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------

def test_alpha_exactly_half_is_wet():
    c = cases.column_case(ny=8, level=0.43)
    j = np.argsort(c.C[1])
    c.alpha = np.where(c.C[1] < 0.4, 1.0, 0.0)
    c.alpha[j[3]] = 0.5  # exact tie
    fc = oracle.faces(c)
    f = [k for k in range(c.F) if {c.owner[k], c.neighbour[k]} == {j[3], j[4]}][0]
    assert fc.kind[f] == 2  # interface, owner (the tie cell) wet
    assert fc.lam[f] == 0.0  # interface sits on the wet cell centre
    p, fc, sy, info = oracle.solve(c, direct=True)
    assert np.all(np.isfinite(p))


def test_unpinned_consistent_system_converges():
    c = cases.box_case(16, 8, 1)
    fc = oracle.faces(c)
    sy = oracle.assemble(c, fc, ref_cell=-1)
    x, it, rel, st = oracle.pcg(sy, rtol=1e-12)
    assert st == 0
    xp, _, _, _ = oracle.solve(c, direct=True)
    d = x - xp
    assert np.ptp(d) <= 1e-8 * np.abs(xp).max()  # differs by a constant only


# --------------------------------------------------------------------------
# planted mistakes: each must break at least one pin
# --------------------------------------------------------------------------

def _still_pin_error(mutate):
    """Largest violation of the still-water pin: corrected flux / jump scale,
    and the distance of the inferred continuity height of the physical
    pressure from the wet-dry cell-centre interval (0 when inside)."""
    c = _still(permute_seed=3)
    p, fc, sy, _ = oracle.solve(c, direct=True, mutate=mutate)
    fcg = oracle.faces(c)
    flux = np.max(np.abs(oracle.corrected_flux(c, fc, p))) / np.max(np.abs(fcg.gamma * fcg.jump))
    wet = c.alpha >= 0.5
    y_gamma = (p[~wet].mean() - p[wet].mean()) / ((c.rho_w - c.rho_a) * c.g[1])
    yW = c.C[1, wet].max()
    yD = c.C[1, ~wet].min()
    outside = max(yW - y_gamma, y_gamma - yD, 0.0)
    return max(flux, outside)


def _ghost_mismatch(mutate):
    c = cases.box_case(10, 8, 3, permute=True, alpha_noise=0.2)
    fc = oracle.faces(c, mutate=mutate)
    p = np.random.default_rng(9).normal(size=c.n) * 1e3
    qp, qm, qg, _, _ = oracle.ghost_route(c, p)
    flux = fc.gamma * ((p[c.neighbour] - p[c.owner]) - fc.jump)
    ok = np.isfinite(qg)
    return np.max(np.abs(qg[ok] - flux[ok])) / np.abs(flux).max()


@pytest.mark.parametrize("mut", [oracle.MUT_JUMP_SIGN_EQ15, oracle.MUT_DROP_JUMP])
def test_planted_jump_mistakes_fail_still_water(mut):
    assert _still_pin_error(oracle.MUT_NONE) <= 1e-12
    assert _still_pin_error(mut) > 1e-3


@pytest.mark.parametrize("mut", [oracle.MUT_LAMBDA_FROM_OWNER, oracle.MUT_ARITH_BETA, oracle.MUT_JUMP_SIGN_EQ15])
def test_planted_coefficient_mistakes_fail_ghost_route(mut):
    assert _ghost_mismatch(oracle.MUT_NONE) <= 1e-9
    assert _ghost_mismatch(mut) > 1e-4


def test_planted_adjoint_mistake_fails_fd():
    c = cases.box_case(16, 8, 1, alpha_noise=0.05, seed=21)
    w = _band_loss_grad(c)
    _, da_ok, _, _ = oracle.adjoint(c, w, direct=True)
    _, da_bad, _, _ = oracle.adjoint(c, w, direct=True, mutate=oracle.MUT_SWAP_ALPHA_DERIV)
    assert np.max(np.abs(da_ok - da_bad)) > 1e-2 * np.abs(da_ok).max()
