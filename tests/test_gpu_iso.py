"""gfm_iso_advect (isoAdvector advection step, Sec. 3.2) against the
oracle through the C ABI.  The kernel sweeps each apex triangle in the
paper's way (ordered vertex times, the cut point x4, two quadratic pieces,
exact integrals); the oracle clips the triangle with the moving half-space
and integrates by Gauss-Legendre between breakpoints: different routes, so
the bar is rounding (1e-12 of dt on the time integrals, 1e-12 on alpha).
Cases: random planar interfaces moving at random normal speeds (both signs,
and static) through a graded 3D mesh and through the non-planar faces of a
distorted 2D mesh; a flat interface carried across cell rows (exact
transport) on a permuted mesh.
"""
import numpy as np
import pytest
import torch

import cases
import oracle

pytestmark = pytest.mark.gpu


def _g():
    import paper_1804_01130_gb300 as g
    return g


def _random_iso(c, seed, frac=0.5, static=False):
    rng = np.random.default_rng(seed)
    has = (rng.random(c.n) < frac).astype(np.int8)
    xS = c.C + rng.uniform(-0.3, 0.3, (3, c.n)) * np.cbrt(c.V)[None]
    nS = rng.normal(size=(3, c.n))
    nS /= np.linalg.norm(nS, axis=0)[None]
    UnS = np.zeros(c.n) if static else rng.uniform(-0.6, 0.6, c.n)
    phi = rng.uniform(-1.0, 1.0, c.F) * np.linalg.norm(c.Sf, axis=0)
    return has, xS, nS, UnS, phi


def _compare(c, has, xS, nS, UnS, phi, dt, renumber=1):
    s = _g().GFM.from_case(c, renumber=renumber)
    dV, I, a_new = s.iso_advect(c.alpha, phi, dt, c.fv_ptr, c.fv_xyz, c.xf, has, xS, nS, UnS, V=c.V)
    I_ref, dV_ref = oracle.iso_flux(c, phi, dt, c.fv_ptr, c.fv_xyz, has, xS, nS, UnS)
    a_ref = oracle.iso_advect(c, dV_ref)
    assert np.max(np.abs(I.cpu().numpy() - I_ref)) <= 1e-12 * dt
    assert np.max(np.abs(dV.cpu().numpy() - dV_ref)) <= 1e-12 * dt * np.max(np.abs(phi))
    assert np.max(np.abs(a_new.cpu().numpy() - a_ref)) <= 1e-11
    return a_new.cpu().numpy()


@pytest.mark.parametrize("seed,static", [(1, False), (2, False), (3, True)])
def test_random_interfaces_on_a_graded_3d_mesh(seed, static):
    rng = np.random.default_rng(seed)
    m = cases.graded_mesh(np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.2, 10))]),
                          np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.2, 8))]),
                          np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.2, 6))]))
    c = cases._case_from(m, rng.random(m["n"]), np.zeros(m["F"]), "g3", (0, 7, 0))
    _compare(c, *_random_iso(c, seed, static=static), dt=0.35)


@pytest.mark.parametrize("renumber", [0, 1])
def test_random_interfaces_on_non_planar_faces(renumber):
    m = cases.wavy_mesh(24, 12, eps=0.06)
    # lift the far corners of every face out of plane
    rng = np.random.default_rng(7)
    m["fv_xyz"] = m["fv_xyz"] + rng.uniform(-0.01, 0.01, m["fv_xyz"].shape)
    c = cases._case_from(m, rng.random(m["n"]), np.zeros(m["F"]), "wavy", (0, 11, 0))
    _compare(c, *_random_iso(c, 8, frac=0.7), dt=0.05, renumber=renumber)


def test_flat_interface_transport_on_a_permuted_mesh():
    nx, ny, level, v, dt = 16, 8, 0.49, 0.5, 0.05
    m = cases.graded_mesh(np.linspace(0.0, 2.0, nx + 1), np.linspace(0.0, 1.0, ny + 1), [0.0, 0.25])
    dy = 1.0 / ny
    alpha = np.clip((level - (m["C"][1] - 0.5 * dy)) / dy, 0.0, 1.0)
    perm = np.random.default_rng(3).permutation(m["n"])
    pm = cases.permute_mesh(m, perm)
    a_p = np.empty_like(alpha)
    a_p[perm] = alpha
    c = cases._case_from(pm, a_p, np.zeros(pm["F"]), "row", (0, ny - 1, 0))
    u = np.array([0.3, v, 0.0])
    phi = u @ c.Sf
    has = ((c.alpha > 0.0) & (c.alpha < 1.0)).astype(np.int8)
    xS = np.stack([c.C[0], np.full(c.n, level), c.C[2]])
    nS = np.zeros((3, c.n))
    nS[1] = 1.0
    a_new = _compare(c, has, xS, nS, np.full(c.n, v), phi, dt)
    expect = np.clip((level + v * dt - (c.C[1] - 0.5 * dy)) / dy, 0.0, 1.0)
    cnt = np.zeros(c.n)
    np.add.at(cnt, c.owner, 1)
    np.add.at(cnt, c.neighbour, 1)
    inner = cnt == 4
    assert np.max(np.abs(a_new - expect)[inner]) <= 1e-12
    assert abs(np.sum(c.V * a_new) - np.sum(c.V * c.alpha)) <= 1e-13
