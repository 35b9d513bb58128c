"""Pins of the oracle's dynamic-pressure gradient (Gauss theorem with the
ghost values of Eq. 20 at interface faces) and of its flux-to-velocity
reconstruction, against what the jump conditions and the mathematics fix.

- A p_d that is linear in each phase and satisfies the jump conditions at
  the interface location of Eqs. 12-13 (Eq. 7: [p_d] = (rho_w - rho_a) g.x;
  Eq. 8: [grad p_d / rho] = 0) is reproduced exactly by the ghost values, so
  (1/rho) grad p_d equals its closed form in every cell (walls carry
  zero-gradient p_d, which halves the wall-normal component there).
- Still water: the solved p_d gives a zero gradient everywhere (the
  balanced-force property stated after Eq. 20).
- One phase: the Gauss gradient of a linear field is exact, on uniform and on
  graded meshes (the face centres set the interpolation weights).
- The reconstruction returns a uniform velocity exactly and converges at
  second order for a divergence-free field tangential to the walls.
Planted mistakes (jump sign of Eq. 15, no jump, the wrong inverse density in
the ghost value, midpoint weights on a graded mesh)
fail them.
"""
import math

import numpy as np
import pytest

import cases
import oracle


def _case(mesh, alpha, name="t"):
    return cases._case_from(mesh, alpha, np.zeros(mesh["F"]), name, (0, mesh["dims"][1] - 1, 0))


def _faces_per_axis(c):
    """Internal faces of each cell along each axis (0, 1 or 2)."""
    cnt = np.zeros((3, c.n))
    ax = np.argmax(np.abs(c.Sf), axis=0)
    np.add.at(cnt, (ax, c.owner), 1)
    np.add.at(cnt, (ax, c.neighbour), 1)
    return cnt


def _two_phase_linear(c, a_y, K_w=123.0):
    """p_d linear in each phase: grad p_w = rho_w a, grad p_a = rho_a a with
    a = (0, a_y, 0), and the jump of Eq. 7 at the Eq. 12-13 interface of a
    flat surface (all interface faces share one lambda)."""
    fc = oracle.faces(c)
    itf = fc.kind >= 2
    assert itf.any()
    o, nb = c.owner[itf], c.neighbour[itf]
    wet_o = c.alpha[o] >= 0.5
    W = np.where(wet_o, o, nb)
    D = np.where(wet_o, nb, o)
    yg = c.C[1, W] + fc.lam[itf] * (c.C[1, D] - c.C[1, W])
    assert np.ptp(yg) < 1e-12  # a plane interface
    y_gamma = float(yg[0])
    g_y = c.g[1]
    # p_a - p_w = (rho_w - rho_a) g.x at x_Gamma with p = rho a.x + K
    K_a = K_w + (c.rho_w - c.rho_a) * (a_y + g_y) * y_gamma
    wet = c.alpha >= 0.5
    return np.where(wet, c.rho_w * a_y * c.C[1] + K_w, c.rho_a * a_y * c.C[1] + K_a)


@pytest.mark.parametrize("nz,permute", [(1, None), (1, 5), (3, None)])
def test_piecewise_linear_field_with_the_jump_has_its_exact_gradient(nz, permute):
    c = cases.still_water_case(nx=16, ny=8, nz=nz, level=0.4475)
    if permute is not None:
        mesh = dict(n=c.n, F=c.F, owner=c.owner, neighbour=c.neighbour, Sf=c.Sf, C=c.C, V=c.V, xf=c.xf,
                    dims=c.dims)
        perm = np.random.default_rng(permute).permutation(c.n)
        pm = cases.permute_mesh(mesh, perm)
        alpha = np.empty_like(c.alpha)
        alpha[perm] = c.alpha
        c = _case(pm, alpha)
    a_y = 3.0
    p = _two_phase_linear(c, a_y)
    G = oracle.gradient(c, p)
    cnt = _faces_per_axis(c)
    expect_y = a_y * cnt[1] / 2.0  # a full cell: a_y; a cell against a wall: a_y / 2
    assert np.max(np.abs(G[1] - expect_y)) <= 1e-8
    assert np.max(np.abs(G[0])) <= 1e-8 and np.max(np.abs(G[2])) <= 1e-8


@pytest.mark.parametrize("mut", [oracle.MUT_JUMP_SIGN_EQ15, oracle.MUT_DROP_JUMP, oracle.MUT_GHOST_SWAP_BETA])
def test_planted_ghost_mistakes_fail_the_piecewise_linear_pin(mut):
    """The jump of Eq. 15 as printed (opposite sign), no jump, or the wet
    side's ghost weighted by the wrong inverse density: the gradient at the
    interface cells is off by O(g)."""
    c = cases.still_water_case(nx=16, ny=8, level=0.4475)
    a_y = 3.0
    p = _two_phase_linear(c, a_y)
    G_bad = oracle.gradient(c, p, mutate=mut)
    cnt = _faces_per_axis(c)
    assert np.max(np.abs(G_bad[1] - a_y * cnt[1] / 2.0)) > 1.0


@pytest.mark.parametrize("nz,permute", [(1, None), (3, None), (1, 9)])
def test_still_water_gradient_vanishes(nz, permute):
    c = cases.still_water_case(nx=16, ny=8, nz=nz, level=0.4475)
    if permute is not None:
        mesh = dict(n=c.n, F=c.F, owner=c.owner, neighbour=c.neighbour, Sf=c.Sf, C=c.C, V=c.V, xf=c.xf,
                    dims=c.dims)
        perm = np.random.default_rng(permute).permutation(c.n)
        pm = cases.permute_mesh(mesh, perm)
        alpha = np.empty_like(c.alpha)
        alpha[perm] = c.alpha
        c = _case(pm, alpha)
    p, _, _, _ = oracle.solve(c, direct=True)
    G = oracle.gradient(c, p)
    # p_d ~ 1e3-1e4 Pa across cells of 0.125 m: rounding of the face sums only
    assert np.max(np.abs(G)) <= 1e-9 * np.max(np.abs(p))


def _graded(nx=9, ny=7, nz=4, seed=2):
    rng = np.random.default_rng(seed)
    xn = np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.3, nx))])
    yn = np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.3, ny))])
    zn = np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.3, nz))])
    return cases.graded_mesh(xn, yn, zn)


@pytest.mark.parametrize("graded", [False, True])
def test_single_phase_linear_field_gradient_is_exact(graded):
    mesh = _graded() if graded else cases.structured_mesh(7, 5, 4, 1.4, 1.0, 0.8)
    c = _case(mesh, np.ones(mesh["n"]))
    a = np.array([1.3, -2.1, 0.7])
    p = c.rho_w * (a @ c.C) + 17.0
    G = oracle.gradient(c, p)
    cnt = _faces_per_axis(c)
    if graded:
        # a wall cell's missing face value sits off the cell centre by an
        # uneven half-width: compare interior cells only
        inner = (cnt == 2).all(axis=0)
        assert inner.sum() > 10
        assert np.max(np.abs(G[:, inner] - a[:, None])) <= 1e-9
        # planted: midpoint weights on the graded mesh are not exact
        G_mid = oracle.gradient(c, p, use_xf=False)
        assert np.max(np.abs(G_mid[:, inner] - a[:, None])) > 1e-2
    else:
        assert np.max(np.abs(G - a[:, None] * cnt / 2.0)) <= 1e-9


def test_reconstruct_returns_a_uniform_velocity():
    for mesh in (cases.structured_mesh(6, 5, 4, 1.2, 1.0, 0.8), _graded()):
        c = _case(mesh, np.ones(mesh["n"]))
        u = np.array([0.3, -0.2, 0.5])
        phi = u @ c.Sf
        U = oracle.reconstruct(c, phi)
        inner = (_faces_per_axis(c) == 2).all(axis=0)
        assert np.max(np.abs(U[:, inner] - u[:, None])) <= 1e-13


def _stream_case(nx, ny, lx=2.0, ly=1.0):
    """psi = sin(pi x/lx) sin(pi y/ly): u = (dpsi/dy, -dpsi/dx), zero normal
    velocity on every wall; face fluxes are exact integrals (psi differences)."""
    mesh = cases.structured_mesh(nx, ny, 1, lx, ly, lx / nx)
    dx, dy, dz = mesh["spacing"]
    psi = lambda x, y: np.sin(math.pi * x / lx) * np.sin(math.pi * y / ly)
    xf, Sf = mesh["xf"], mesh["Sf"]
    xface = np.abs(Sf[0]) > 0
    phi = np.where(xface, dz * (psi(xf[0], xf[1] + dy / 2) - psi(xf[0], xf[1] - dy / 2)),
                   -dz * (psi(xf[0] + dx / 2, xf[1]) - psi(xf[0] - dx / 2, xf[1])))
    c = _case(mesh, np.ones(mesh["n"]))
    x, y = c.C[0], c.C[1]
    u = np.stack([math.pi / ly * np.sin(math.pi * x / lx) * np.cos(math.pi * y / ly),
                  -math.pi / lx * np.cos(math.pi * x / lx) * np.sin(math.pi * y / ly)])
    return c, phi, u


def test_reconstruct_converges_at_second_order():
    errs = []
    for nx, ny in ((16, 8), (32, 16), (64, 32)):
        c, phi, u = _stream_case(nx, ny)
        U = oracle.reconstruct(c, phi)
        errs.append(np.max(np.abs(U[:2] - u)))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
