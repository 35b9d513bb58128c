"""Pins of the oracle's isoAdvector advection step (Sec. 3.2): the face
integral I_f = int_0^dt alpha_f+(tau) dtau of a planar interface moving at
constant normal speed, and the volume-fraction update.

- Closed forms on a unit square face: an interface parallel to an edge
  (alpha_f+ linear in tau, both directions of motion, with and without the
  face filling up within the step) and one along the diagonal (quadratic
  pieces).
- Reversing the interface's orientation and speed gives the complement:
  I(n, U) + I(-n, -U) = dt.
- Monte Carlo sampling of the submerged area of a non-planar quadrilateral
  (the union of its four apex triangles, as the paper defines the surface).
- The update conserves the heavy-fluid volume and moves a flat interface by
  exactly u dt, within its row of cells and across into the next row.
A planted mistake (the downwind cell's interface) fails the pins.
"""
import math

import numpy as np
import pytest

import cases
import oracle


def _two_cells(length=1.0):
    """Cells [0,1] and [1,2] x [0,1] x [0,1]: one internal face, the unit square at x = 1."""
    m = cases.graded_mesh([0.0, 1.0, 2.0], [0.0, length], [0.0, length])
    return cases._case_from(m, np.array([0.5, 0.0]), np.zeros(1), "two", (0, 0, 0))


def _iso(c, xs, ns, un, phi=1.0, dt=1.0, has=(1, 0)):
    xS = np.zeros((3, c.n))
    nS = np.zeros((3, c.n))
    UnS = np.zeros(c.n)
    xS[:, 0] = xs
    nS[:, 0] = np.asarray(ns) / np.linalg.norm(ns)
    UnS[0] = un
    I, dV = oracle.iso_flux(c, np.array([phi]), dt, c.fv_ptr, c.fv_xyz, np.array(has, dtype=np.int8), xS, nS, UnS)
    return float(I[0]), float(dV[0])


@pytest.mark.parametrize("un,dt,expect", [
    (0.5, 1.0, 0.55),             # 0.3 + 0.5 tau, never full
    (0.5, 2.0, 0.91 + 0.6),       # full at tau = 1.4
    (-0.2, 2.0, 0.225),           # draining: empty at tau = 1.5
    (0.0, 1.5, 0.45),             # static interface
])
def test_interface_parallel_to_an_edge(un, dt, expect):
    c = _two_cells()
    I, dV = _iso(c, (0.5, 0.3, 0.5), (0.0, 1.0, 0.0), un, phi=2.0, dt=dt)
    assert abs(I - expect) <= 1e-13
    assert abs(dV - 2.0 * expect) <= 2e-13


def test_interface_along_the_diagonal():
    c = _two_cells()
    # heavy where y + z < 1 + tau (unit-speed along (0,1,1)/sqrt 2 scaled): area
    # fraction 1 - (1 - tau)^2 / 2 on [0, 1]
    I, _ = _iso(c, (1.0, 0.5, 0.5), (0.0, 1.0, 1.0), 1.0 / math.sqrt(2.0), dt=1.0)
    assert abs(I - 5.0 / 6.0) <= 1e-13
    # starting below: c = 0.4 + tau, crosses the corner at tau = 0.6
    I, _ = _iso(c, (1.0, 0.2, 0.2), (0.0, 1.0, 1.0), 1.0 / math.sqrt(2.0), dt=1.0)
    # int_0^0.6 (0.4 + t)^2 / 2 dt + int_0.6^1 [1 - (1.6 - t)^2 / 2] dt
    a = (1.0 ** 3 - 0.4 ** 3) / 6.0
    b = 0.4 - (1.0 ** 3 - 0.6 ** 3) / 6.0
    assert abs(I - (a + b)) <= 1e-13, (I, a + b)


def _random_quad_case(seed):
    """Two hexahedral cells sharing a non-planar quadrilateral face."""
    rng = np.random.default_rng(seed)
    c = _two_cells()
    quad = np.array([[1.0, 0.0, 0.0], [1.0, 1.0, 0.0], [1.0, 1.0, 1.0], [1.0, 0.0, 1.0]]).T
    quad = quad + rng.uniform(-0.15, 0.15, quad.shape)
    c.fv_xyz = np.ascontiguousarray(quad)
    c.xf = quad.mean(axis=1).reshape(3, 1)
    return c, rng


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_reversed_interface_gives_the_complement(seed):
    c, rng = _random_quad_case(seed)
    xs = rng.uniform(0.7, 1.3, 3)
    ns = rng.normal(size=3)
    un = rng.uniform(-0.4, 0.4)
    dt = 1.3
    I1, _ = _iso(c, xs, ns, un, dt=dt)
    I2, _ = _iso(c, xs, -np.asarray(ns), -un, dt=dt)
    assert abs(I1 + I2 - dt) <= 1e-12


def _monte_carlo(c, xs, ns, un, dt, samples=20000, steps=400, seed=0):
    rng = np.random.default_rng(seed)
    apex = c.xf[:, 0]
    quad = c.fv_xyz
    pts, wts = [], []
    for e in range(4):
        a, b = quad[:, e], quad[:, (e + 1) % 4]
        area = 0.5 * np.linalg.norm(np.cross(a - apex, b - apex))
        r1, r2 = rng.random(samples), rng.random(samples)
        s = np.sqrt(r1)
        p = (1 - s)[None] * apex[:, None] + (s * (1 - r2))[None] * a[:, None] + (s * r2)[None] * b[:, None]
        pts.append(p)
        wts.append(np.full(samples, area / samples))
    P, W = np.concatenate(pts, axis=1), np.concatenate(wts)
    n = np.asarray(ns) / np.linalg.norm(ns)
    d = (P - np.asarray(xs)[:, None]).T @ n
    taus = (np.arange(steps) + 0.5) * dt / steps
    frac = [(W * (d < un * t)).sum() / W.sum() for t in taus]
    return float(np.sum(frac) * dt / steps)


@pytest.mark.parametrize("seed", [4, 5])
def test_monte_carlo_on_a_non_planar_face(seed):
    c, rng = _random_quad_case(seed)
    xs = np.array([1.0, 0.35, 0.4])
    ns = np.array([0.1, 1.0, 0.6]) + rng.uniform(-0.2, 0.2, 3)
    un, dt = 0.3, 1.2
    I, _ = _iso(c, xs, ns, un, dt=dt)
    assert abs(I - _monte_carlo(c, xs, ns, un, dt)) <= 6e-3


def _row_case(nx=12, ny=8, level=0.44):
    """A flat interface inside one row of cells on the 2 x 1 box."""
    m = cases.graded_mesh(np.linspace(0.0, 2.0, nx + 1), np.linspace(0.0, 1.0, ny + 1), [0.0, 0.25])
    dy = 1.0 / ny
    alpha = np.clip((level - (m["C"][1] - 0.5 * dy)) / dy, 0.0, 1.0)
    return cases._case_from(m, alpha, np.zeros(m["F"]), "row", (0, ny - 1, 0)), dy


def _interior(c):
    """Cells with all four in-plane neighbours (none against a wall)."""
    cnt = np.zeros(c.n)
    np.add.at(cnt, c.owner, 1)
    np.add.at(cnt, c.neighbour, 1)
    return cnt == 4


def _flat_iso(c, level, v):
    cut = (c.alpha > 0.0) & (c.alpha < 1.0)
    xS = np.zeros((3, c.n))
    xS[0], xS[1], xS[2] = c.C[0], level, c.C[2]
    nS = np.zeros((3, c.n))
    nS[1] = 1.0
    return cut.astype(np.int8), xS, nS, np.full(c.n, v)


@pytest.mark.parametrize("v,level,dt", [
    (0.5, 0.44, 0.01), (-0.5, 0.44, 0.01),   # the interface stays inside its row
    (0.5, 0.49, 0.05), (-0.5, 0.38, 0.05),   # it crosses into the next row during the step
])
def test_flat_interface_moves_by_u_dt(v, level, dt):
    c, dy = _row_case(level=level)
    u = np.array([0.3, v, 0.0])
    phi = u @ c.Sf
    has, xS, nS, UnS = _flat_iso(c, level, v)
    I, dV = oracle.iso_flux(c, phi, dt, c.fv_ptr, c.fv_xyz, has, xS, nS, UnS)
    a_new = oracle.iso_advect(c, dV)
    expect = np.clip((level + v * dt - (c.C[1] - 0.5 * dy)) / dy, 0.0, 1.0)
    # a uniform velocity crosses the walls, which carry no flux: compare the
    # cells away from them
    inner = _interior(c)
    assert np.max(np.abs(a_new - expect)[inner]) <= 1e-12
    # heavy-fluid volume conserved: internal faces cancel
    assert abs(np.sum(c.V * a_new) - np.sum(c.V * c.alpha)) <= 1e-14


def test_planted_downwind_interface_fails():
    """Taking the interface from the downwind cell moves the flat
    interface by the wrong amount."""
    level, v, dt = 0.49, 0.5, 0.05
    c, dy = _row_case(level=level)
    u = np.array([0.0, v, 0.0])
    phi = u @ c.Sf
    has, xS, nS, UnS = _flat_iso(c, level, v)
    I, dV = oracle.iso_flux(c, phi, dt, c.fv_ptr, c.fv_xyz, has, xS, nS, UnS, mutate=oracle.MUT_ISO_DOWNWIND)
    a_new = oracle.iso_advect(c, dV)
    expect = np.clip((level + v * dt - (c.C[1] - 0.5 * dy)) / dy, 0.0, 1.0)
    assert np.max(np.abs(a_new - expect)[_interior(c)]) > 1e-2
