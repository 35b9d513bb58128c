"""GPU parity: libgfm (through its C ABI) against the CPU FP64 oracle.

Bars: assembly (lambda, gamma, J, diag, b) bit-exact in FP64; p_d within
relative L2 1e-9 (FP64 mode) and 1e-6 (mixed mode) of the oracle.  Cases
span several 32-cell slices with a ragged tail, 2D and 3D, caller order,
random permutations, and the three renumberings.
"""
import numpy as np
import pytest
import torch

import cases
import oracle

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
MIXED_TOL = 1e-6


def _gfm():
    import paper_1804_01130_gb300 as g
    return g


def _setup(case, renumber=1):
    g = _gfm()
    s = g.GFM.from_case(case, renumber=renumber)
    s.assemble(torch.as_tensor(case.alpha), torch.as_tensor(case.phi), case.rho_w, case.rho_a, case.g, case.ref_cell,
               case.ref_value)
    return s


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SMALL = {
    "tank_8x4": lambda: cases.box_case(8, 4, 1, seed=3, ka=0.15),
    "config1_64x32": lambda: cases.make_case(1),
    "tank_37x19_ragged": lambda: cases.box_case(37, 19, 1, seed=8, nwaves=2),
    "box_12x10x5_perm": lambda: cases.box_case(12, 10, 5, seed=4, permute=True, alpha_noise=0.1),
    "column_1x40": lambda: cases.column_case(ny=40, level=0.5173),
}


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("renumber", [0, 1, 2])
def test_assembly_bit_exact(name, renumber):
    c = SMALL[name]()
    s = _setup(c, renumber)
    ex = {k: v.cpu().numpy() for k, v in s.export_system().items()}
    fc = oracle.faces(c)
    sy = oracle.assemble(c, fc)
    assert np.array_equal(ex["lambda"], fc.lam)
    assert np.array_equal(ex["gamma"], fc.gamma)
    assert np.array_equal(ex["jump"], fc.jump)
    assert np.array_equal(ex["diag"], sy.diag)
    assert np.array_equal(ex["b"], sy.b)


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("mode,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_solve_matches_oracle(name, mode, tol):
    c = SMALL[name]()
    p_ref, fc, sy, _ = oracle.solve(c, direct=c.n <= 2048, rtol=1e-14)
    s = _setup(c)
    p, _, info = s.solve(mode=mode, rtol=1e-13 if mode == "fp64" else 1e-12)
    assert info.status == 0, info
    assert info.rel_res_l2 <= 1e-12
    err = _rel(p.cpu().numpy(), p_ref)
    assert err <= tol, (err, info)
    # the dynamic part alone (the hydrostatic jump offset dominates ||p||)
    p_still, _, _, _ = oracle.solve(c, direct=c.n <= 2048, rtol=1e-14, phi=np.zeros(c.F))
    dyn_ref = p_ref - p_still
    s.assemble(torch.as_tensor(c.alpha), torch.zeros(c.F, dtype=torch.float64), c.rho_w, c.rho_a, c.g, c.ref_cell)
    ps, _, _ = s.solve(mode=mode, rtol=1e-13 if mode == "fp64" else 1e-12)
    dyn = p.cpu().numpy() - ps.cpu().numpy()
    assert _rel(dyn, dyn_ref) <= 1e3 * tol


@pytest.mark.parametrize("renumber", [0, 1, 2])
def test_renumberings_agree(renumber):
    c = cases.box_case(20, 12, 3, seed=9, permute=True)
    p_ref, _, _, _ = oracle.solve(c, direct=False, rtol=1e-14)
    s = _setup(c, renumber)
    p, _, info = s.solve(mode="fp64", rtol=1e-13)
    assert info.status == 0
    assert _rel(p.cpu().numpy(), p_ref) <= FP64_TOL
    perm = s.permutation()
    assert np.array_equal(np.sort(perm), np.arange(c.n))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_corrected_flux_and_still_water(mode):
    c = cases.still_water_case(nx=40, ny=20, level=0.4475)
    s = _setup(c)
    p, fcorr, info = s.solve(mode=mode, rtol=1e-13, phi_corr=True)
    assert info.status == 0
    fc = oracle.faces(c)
    scale = np.max(np.abs(fc.gamma * fc.jump))
    assert np.max(np.abs(fcorr.cpu().numpy())) <= 1e-10 * scale
    wet = c.alpha >= 0.5
    pn = p.cpu().numpy()
    assert np.ptp(pn[wet]) <= 1e-9 * np.abs(pn).max()
    # corrected flux matches the oracle's on a flow case
    c2 = cases.make_case(1)
    s2 = _setup(c2)
    p2, f2, _ = s2.solve(mode=mode, rtol=1e-13, phi_corr=True)
    fo = oracle.corrected_flux(c2, oracle.faces(c2), p2.cpu().numpy())
    assert np.max(np.abs(f2.cpu().numpy() - fo)) <= 1e-12 * np.abs(fo).max()


def test_golden_fixtures_on_gpu():
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_golden
    for name in make_golden.FIXTURES:
        c, gold = make_golden.case(name)
        s = _setup(c)
        ex = {k: v.cpu().numpy() for k, v in s.export_system().items()}
        for k in ("lambda", "gamma", "jump", "diag", "b"):
            assert np.array_equal(ex[k], gold[k]), (name, k)
        p, fcorr, info = s.solve(mode="fp64", rtol=1e-14, phi_corr=True)
        assert _rel(p.cpu().numpy(), gold["p"]) <= FP64_TOL
        p, fcorr, info = s.solve(mode="mixed", rtol=1e-13, phi_corr=True)
        assert _rel(p.cpu().numpy(), gold["p"]) <= MIXED_TOL
