"""Pins of the oracle's real pressure-equation inputs (Sec. 3): a face
Rhie-Chow coefficient rau_f (1/a_P of the momentum equation) in the face
coefficient, and the explicit over-relaxed non-orthogonal correction with its
deferred-correction loop.

- Balanced force survives any positive rau field: still water stays still,
  with the hydrostatic jump (Eqs. 3, 7).
- A uniform rau = r with the predicted flux scaled by r leaves p_d unchanged.
- On orthogonal meshes the correction vanishes (S_f parallel to d_f).
- On a smoothly distorted mesh a manufactured Neumann problem converges
  under refinement only with the correction; without it the error stays at
  O(1) (the two-point flux is inconsistent when S_f is not parallel to d_f).
A planted sign error in the correction fails the last pin.
"""
import math

import numpy as np
import pytest

import cases
import oracle


def test_still_water_stays_still_for_any_rau():
    c = cases.still_water_case(nx=16, ny=8, level=0.4475)
    rau = np.random.default_rng(3).uniform(0.5, 2.0, c.F)
    fc = oracle.faces(c, rau=rau)
    sy = oracle.assemble(c, fc)
    p = oracle.cholesky_solve(sy)
    q = oracle.corrected_flux(c, fc, p)
    assert np.max(np.abs(q)) <= 1e-12 * np.max(np.abs(fc.gamma * fc.jump))
    wet = c.alpha >= 0.5
    assert np.ptp(p[wet]) <= 1e-9 * np.max(np.abs(p)) and np.ptp(p[~wet]) <= 1e-9 * np.max(np.abs(p))
    # the jump of Eq. 7 at every interface face
    itf = fc.kind >= 2
    assert np.allclose(p[c.neighbour[itf]] - p[c.owner[itf]], fc.jump[itf], rtol=1e-11, atol=0)


def test_rau_enters_the_face_coefficient():
    c = cases.box_case(12, 8, 1, seed=2, ka=0.12)
    rau = np.random.default_rng(5).uniform(0.5, 2.0, c.F)
    f1, fr = oracle.faces(c), oracle.faces(c, rau=rau)
    assert np.array_equal(fr.gamma, f1.gamma * rau)
    assert np.array_equal(fr.jump, f1.jump) and np.array_equal(fr.lam, f1.lam)


@pytest.mark.parametrize("r", [0.25, 3.0])
def test_uniform_rau_with_scaled_flux_leaves_p_unchanged(r):
    c = cases.box_case(16, 10, 1, seed=8, ka=0.1)
    p1 = oracle.cholesky_solve(oracle.assemble(c, oracle.faces(c)))
    fr = oracle.faces(c, rau=np.full(c.F, r))
    pr = oracle.cholesky_solve(oracle.assemble(c, fr, phi=r * c.phi))
    assert np.linalg.norm(pr - p1) <= 1e-11 * np.linalg.norm(p1)


def test_correction_vanishes_on_orthogonal_meshes():
    c = cases.box_case(16, 10, 3, seed=4, ka=0.1, permute=True)
    p, _, _, _ = oracle.solve(c, direct=False, rtol=1e-12)
    corr = oracle.nonorth_correction(c, p)
    scale = np.max(np.abs(oracle.faces(c).gamma * (p[c.neighbour] - p[c.owner])))
    assert np.max(np.abs(corr)) <= 1e-13 * scale


def _mms(nx, corrs, mutate=oracle.MUT_NONE):
    """-div(beta grad p) = f on the distorted mesh of a 2 x 1 rectangle with
    p = cos(pi x/2) cos(pi y): zero normal gradient on the walls; the face
    source is the exact face flux beta S_f . grad p(x_f)."""
    ny = nx // 2
    m = cases.wavy_mesh(nx, ny)
    pex = lambda x, y: np.cos(math.pi * x / 2.0) * np.cos(math.pi * y)
    gx = lambda x, y: -math.pi / 2.0 * np.sin(math.pi * x / 2.0) * np.cos(math.pi * y)
    gy = lambda x, y: -math.pi * np.cos(math.pi * x / 2.0) * np.sin(math.pi * y)
    beta = 1.0 / cases.RHO_W
    xf = m["xf"]
    phi = beta * (m["Sf"][0] * gx(xf[0], xf[1]) + m["Sf"][1] * gy(xf[0], xf[1]))
    c = cases._case_from(m, np.ones(m["n"]), phi, "mms", (0, ny - 1, 0))
    c.ref_value = float(pex(c.C[0, c.ref_cell], c.C[1, c.ref_cell]))
    p, _, _, _ = oracle.solve_nonorth(c, corrs, direct=False, rtol=1e-13, mutate=mutate)
    return float(np.max(np.abs(p - pex(c.C[0], c.C[1]))))


def test_manufactured_solution_converges_only_with_the_correction():
    with_c = [_mms(nx, 20) for nx in (16, 32, 64)]
    without = [_mms(nx, 0) for nx in (16, 32, 64)]
    assert with_c[0] / with_c[1] > 1.5 and with_c[1] / with_c[2] > 1.7, with_c
    assert without[2] > 0.9 * without[0]  # no convergence without it
    assert with_c[2] < without[2] / 10.0


def test_planted_correction_sign_fails_the_manufactured_pin():
    bad = [_mms(nx, 8, mutate=oracle.MUT_NONORTH_SIGN) for nx in (16, 32)]
    good = _mms(32, 8)
    assert bad[1] > 5.0 * good
