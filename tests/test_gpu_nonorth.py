"""Real pressure-equation inputs on the GPU against the oracle, through the
C ABI: the face Rhie-Chow coefficient (gfm_set_rau, bit-exact assembly)
and the explicit non-orthogonal correction with its deferred-correction
loop (gfm_nonorth_correct), on a smoothly distorted two-phase mesh.

Bars: assembly with rau bit-exact; the correction flux and the corrected
source within rounding of the oracle's (different but equivalent gradient
formulas: 1e-11 of the largest coefficient flux); deferred-correction
solutions within relative L2 1e-9 (FP64) / 1e-6 (mixed) of the oracle's loop.
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


def _wavy_two_phase(nx=48, ny=24, seed=3):
    m = cases.wavy_mesh(nx, ny)
    dy = 1.0 / ny
    alpha = np.clip((0.45 - m["C"][1]) / dy + 0.5, 0.0, 1.0)
    phi = cases.random_face_flux(m, np.random.default_rng(seed), two_d=True)
    return cases._case_from(m, alpha, phi, "wavy", (0, ny - 1, 0))


def _handle(c, rau=None, renumber=1):
    g = _g()
    s = g.GFM.from_case(c, renumber=renumber)
    if rau is not None:
        s.set_rau(torch.as_tensor(rau))
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    return s


@pytest.mark.parametrize("mk", [lambda: cases.make_case(1), lambda: cases.box_case(12, 10, 5, seed=6, permute=True)])
def test_rau_assembly_is_bit_exact_and_solves(mk):
    c = mk()
    rau = np.random.default_rng(11).uniform(0.5, 2.0, c.F)
    s = _handle(c, rau)
    ex = {k: v.cpu().numpy() for k, v in s.export_system().items()}
    fc = oracle.faces(c, rau=rau)
    sy = oracle.assemble(c, fc)
    for k, ref in (("lambda", fc.lam), ("gamma", fc.gamma), ("jump", fc.jump), ("diag", sy.diag), ("b", sy.b)):
        assert np.array_equal(ex[k], ref), k
    p_ref = oracle.cholesky_solve(sy) if c.n <= 4096 else oracle.pcg(sy, rtol=1e-13)[0]
    for mode, tol in (("fp64", 1e-9), ("mixed", 1e-6)):
        p, _, info = s.solve(mode=mode, rtol=1e-12 if mode == "fp64" else 1e-10)
        assert info.status == 0
        assert np.linalg.norm(p.cpu().numpy() - p_ref) <= tol * np.linalg.norm(p_ref), mode
    # clearing it restores the plain coefficient
    s.set_rau(None)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    assert np.array_equal(s.export_system()["gamma"].cpu().numpy(), oracle.faces(c).gamma)


@pytest.mark.parametrize("use_rau", [False, True])
def test_correction_flux_and_source_match_the_oracle(use_rau):
    c = _wavy_two_phase()
    rau = np.random.default_rng(2).uniform(0.5, 2.0, c.F) if use_rau else None
    s = _handle(c, rau)
    fc = oracle.faces(c, rau=rau)
    p_ref = oracle.cholesky_solve(oracle.assemble(c, fc))
    corr = s.nonorth_correct(torch.as_tensor(p_ref), torch.as_tensor(c.V), xf=torch.as_tensor(c.xf),
                             return_corr=True).cpu().numpy()
    corr_ref = oracle.nonorth_correction(c, p_ref, rau=rau)
    scale = np.max(np.abs(fc.gamma * (p_ref[c.neighbour] - p_ref[c.owner] - fc.jump)))
    assert np.max(np.abs(corr_ref)) > 1e-6 * scale  # the mesh is not orthogonal
    assert np.max(np.abs(corr - corr_ref)) <= 1e-11 * scale
    b = s.export_system()["b"].cpu().numpy()
    b_ref = oracle.assemble(c, fc, phi=c.phi - corr_ref).b
    assert np.max(np.abs(b - b_ref)) <= 1e-11 * np.max(np.abs(b_ref))


@pytest.mark.parametrize("mode,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_deferred_correction_loop_matches_the_oracle(mode, tol):
    c = _wavy_two_phase()
    correctors = 5
    p_ref, corr_ref, fc, _ = oracle.solve_nonorth(c, correctors, direct=True)
    s = _handle(c)
    V, xf = torch.as_tensor(c.V), torch.as_tensor(c.xf)
    rtol = 1e-12 if mode == "fp64" else 1e-10
    p, _, info = s.solve(mode=mode, rtol=rtol)
    assert info.status == 0
    for _ in range(correctors):
        s.nonorth_correct(p, V, xf=xf)
        p, fl, info = s.solve(mode=mode, rtol=rtol, p0=p.clone(), phi_corr=True)
        assert info.status == 0
    pn = p.cpu().numpy()
    assert np.linalg.norm(pn - p_ref) <= tol * np.linalg.norm(p_ref)
    # corrected flux: phi* - corr - gamma (p_nb - p_own - J), with the last correction
    fl_ref = (c.phi - corr_ref) - fc.gamma * ((pn[c.neighbour] - pn[c.owner]) - fc.jump)
    assert np.max(np.abs(fl.cpu().numpy() - fl_ref)) <= 1e-6 * np.max(np.abs(fc.gamma * fc.jump))


def test_correction_is_zero_on_orthogonal_meshes_and_cleared_by_assembly():
    c = cases.box_case(16, 10, 3, seed=4, ka=0.1, permute=True)
    s = _handle(c)
    p, _, _ = s.solve(mode="fp64", rtol=1e-12)
    b0 = s.export_system()["b"].cpu().numpy()
    corr = s.nonorth_correct(p, torch.as_tensor(c.V), return_corr=True).cpu().numpy()
    fc = oracle.faces(c)
    pn = p.cpu().numpy()
    assert np.max(np.abs(corr)) <= 1e-13 * np.max(np.abs(fc.gamma * (pn[c.neighbour] - pn[c.owner])))
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    assert np.array_equal(s.export_system()["b"].cpu().numpy(), b0)
