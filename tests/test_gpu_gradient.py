"""gfm_gradient (GFM dynamic-pressure gradient with the Eq. 20 ghost values,
and the flux-to-velocity reconstruction) against the CPU oracle, through the
C ABI, on the same p_d (the oracle's solution) and the same face flux.

The two sides use different but equivalent formulas: the oracle forms the
ghost values of Eq. 20 literally, the kernel their collapsed form on the
assembled lambda and J, so the bar is rounding, not bits:
|G_gpu - G_oracle| <= 1e-12 * max|p| * max(|S_f|/V) / rho_a (+ the same
relative to |G|).  Cases: the config-1 tank, a ragged tank, a permuted 3D
box, still water, a graded 3D mesh with and without face centres, and a
batched handle.
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


def _scale(c, p):
    sv = np.max(np.linalg.norm(c.Sf, axis=0)) / np.min(c.V)
    return 1e-12 * np.max(np.abs(p)) * sv / c.rho_a


def _check(c, renumber=1, use_xf=True, p=None):
    g = _g()
    s = g.GFM.from_case(c, renumber=renumber)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    if p is None:
        p, fc, sy, _ = oracle.solve(c, direct=c.n <= 1024, rtol=1e-13)
    else:
        fc = oracle.faces(c)
    phi_corr = oracle.corrected_flux(c, fc, p)
    xf = c.xf if use_xf else None
    G, U = s.gradient(torch.as_tensor(p), torch.as_tensor(c.V), xf=None if xf is None else torch.as_tensor(xf),
                      phi=torch.as_tensor(phi_corr))
    G_ref = oracle.gradient(c, p, use_xf=use_xf)
    U_ref = oracle.reconstruct(c, phi_corr, use_xf=use_xf)
    G = G.cpu().numpy()
    U = U.cpu().numpy()
    tol = _scale(c, p) + 1e-12 * np.max(np.abs(G_ref))
    assert np.max(np.abs(G - G_ref)) <= tol, (c.name, np.max(np.abs(G - G_ref)), tol)
    utol = 1e-12 * (np.max(np.abs(phi_corr)) * np.max(np.linalg.norm(c.Sf, axis=0)) / np.min(c.V) + 1e-300)
    assert np.max(np.abs(U - U_ref)) <= utol + 1e-12 * np.max(np.abs(U_ref)), (c.name, np.max(np.abs(U - U_ref)))
    return G, G_ref


@pytest.mark.parametrize("mk", [
    lambda: cases.make_case(1),
    lambda: cases.box_case(37, 19, 1, seed=4, ka=0.15),
    lambda: cases.box_case(12, 10, 5, seed=6, permute=True, alpha_noise=0.05),
])
@pytest.mark.parametrize("renumber", [0, 1, 2])
def test_gradient_matches_oracle(mk, renumber):
    _check(mk(), renumber=renumber)


def test_still_water_gradient_is_zero_on_the_gpu():
    c = cases.still_water_case(nx=16, ny=8, nz=3, level=0.4475)
    p, _, _, _ = oracle.solve(c, direct=True)
    G, _ = _check(c, p=p)
    assert np.max(np.abs(G)) <= 1e-9 * np.max(np.abs(p))


@pytest.mark.parametrize("use_xf", [True, False])
def test_graded_mesh_with_and_without_face_centres(use_xf):
    rng = np.random.default_rng(2)
    mesh = cases.graded_mesh(np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.3, 11))]),
                             np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.3, 9))]),
                             np.concatenate([[0.0], np.cumsum(rng.uniform(0.05, 0.3, 4))]))
    eta = 0.5 * (mesh["C"][1].min() + mesh["C"][1].max())
    dy = mesh["spacing"][1]
    alpha = np.clip((eta - mesh["C"][1]) / dy + 0.5, 0.0, 1.0)
    phi = cases.random_face_flux(mesh, np.random.default_rng(3), two_d=False)
    c = cases._case_from(mesh, alpha, phi, "graded", (0, mesh["dims"][1] - 1, 0))
    _check(c, use_xf=use_xf)


def test_gradient_on_a_batched_handle():
    g = _g()
    tanks = cases.batch_cases(5, seed0=4200, nx_range=(20, 60), ny_range=(8, 30))
    b = g.GFMBatch(tanks, renumber=1)
    alpha = torch.as_tensor(np.concatenate([t.alpha for t in tanks]))
    phi = torch.as_tensor(np.concatenate([t.phi for t in tanks]))
    # a second density pair on one tank: densities are taken per tank
    phys = [dict(rho_w=t.rho_w, rho_a=(t.rho_a if k != 2 else 1.2), g=t.g, ref_cell=t.ref_cell,
                 ref_value=t.ref_value) for k, t in enumerate(tanks)]
    b.assemble(alpha, phi, phys)
    ps, Vs, xfs, refs = [], [], [], []
    for k, t in enumerate(tanks):
        t.rho_a = phys[k]["rho_a"]
        p, _, _, _ = oracle.solve(t, rtol=1e-13, direct=False)
        ps.append(p)
        Vs.append(t.V)
        xfs.append(t.xf)
        refs.append(oracle.gradient(t, p))
    G, _ = b.gradient(torch.as_tensor(np.concatenate(ps)), torch.as_tensor(np.concatenate(Vs)),
                      xf=torch.as_tensor(np.concatenate(xfs, axis=1)))
    G = G.cpu().numpy()
    c0 = 0
    for t, p, G_ref in zip(tanks, ps, refs):
        Gt = G[:, c0:c0 + t.n]
        assert np.max(np.abs(Gt - G_ref)) <= _scale(t, p) + 1e-12 * np.max(np.abs(G_ref)), t.name
        c0 += t.n


def test_gradient_argument_errors():
    g = _g()
    c = cases.box_case(8, 6, 1, seed=1)
    s = g.GFM.from_case(c)
    p = torch.zeros(c.n, dtype=torch.float64, device="cuda")
    V = torch.as_tensor(c.V).cuda()
    with pytest.raises(g.GFMError) as e:
        s.gradient(p, V)  # before assembly
    assert e.value.status == g.GFM_ERR_STATE
    lib = g.load_library()
    assert lib.gfm_gradient(s.h, None, None, None, None, None, None, None) == g.GFM_ERR_ARG
