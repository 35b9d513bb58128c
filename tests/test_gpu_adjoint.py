"""GPU adjoint (reverse mode through solve and assembly) against the CPU
oracle's gradient and against central finite differences of GPU solves."""
import numpy as np
import pytest
import torch

import cases
import oracle

pytestmark = pytest.mark.gpu


def _g():
    import paper_1804_01130_gb300 as g
    return g


def _band(c, x0, x1, y0, y1):
    return np.where((c.C[0] >= x0) & (c.C[0] <= x1) & (c.C[1] >= y0) & (c.C[1] <= y1), c.V, 0.0)


def _setup(c, renumber=1):
    s = _g().GFM.from_case(c, renumber=renumber)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    return s


@pytest.mark.parametrize("name,mk", [
    ("config1", lambda: cases.make_case(1)),
    ("box_perm", lambda: cases.box_case(12, 8, 4, seed=6, permute=True, alpha_noise=0.05)),
])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_adjoint_matches_oracle(name, mk, mode):
    c = mk()
    w = _band(c, 0.5, 1.5, 0.35, 0.65) if c.dims[2] == 1 else np.where(np.abs(c.C[1] - 0.5) < 0.15, c.V, 0.0)
    dphi_ref, dalpha_ref, mu_ref, p_ref = oracle.adjoint(c, w, direct=c.n <= 2048, rtol=1e-14)
    s = _setup(c)
    p, _, _ = s.solve(mode="fp64", rtol=1e-13)
    dphi, dalpha, mu, info = s.adjoint(p, torch.as_tensor(w), mode=mode, rtol=1e-12)
    assert info.status == 0
    scale_mu = np.abs(mu_ref).max()
    assert np.max(np.abs(mu.cpu().numpy() - mu_ref)) <= 1e-7 * scale_mu
    for got, ref in ((dphi, dphi_ref), (dalpha, dalpha_ref)):
        g_ = got.cpu().numpy()
        assert np.max(np.abs(g_ - ref)) <= 1e-5 * np.abs(ref).max()


def test_autograd_function_backward():
    g = _g()
    c = cases.make_case(1)
    s = g.GFM.from_case(c)
    alpha = torch.as_tensor(c.alpha).cuda().requires_grad_(True)
    phi = torch.as_tensor(c.phi).cuda().requires_grad_(True)
    w = torch.as_tensor(_band(c, 0.5, 1.5, 0.35, 0.65)).cuda()
    phys = dict(rho_w=c.rho_w, rho_a=c.rho_a, g=c.g, ref_cell=c.ref_cell)
    # 1e-11: an attainable target for the FP32-inner adjoint of this source
    p = g.GFMSolve.apply(alpha, phi, s, phys, dict(mode="mixed", rtol=1e-11))
    loss = (w * p).sum()
    loss.backward()
    dphi_ref, dalpha_ref, _, _ = oracle.adjoint(c, w.cpu().numpy(), direct=True)
    assert np.max(np.abs(phi.grad.cpu().numpy() - dphi_ref)) <= 1e-5 * np.abs(dphi_ref).max()
    assert np.max(np.abs(alpha.grad.cpu().numpy() - dalpha_ref)) <= 1e-5 * np.abs(dalpha_ref).max()


def test_adjoint_vs_central_differences_tank():
    """Deck-band loss on the 1024x512 tank: 16 face-flux and up to 16 alpha
    entries against central differences of FP64 GPU solves.  phi enters the
    source affinely, so a central difference is exact for any step: the step
    is 100 max|phi|, far above the solves' noise, and the bar is 1e-5.  alpha
    enters through lambda, gamma and J nonlinearly, and L ~ 50 carries ~5e-11
    of solve noise: Richardson-extrapolated central differences (h = 4e-3 and
    2e-3, error O(h^4)) on the entries of at least a fifth of max|dL/dalpha|,
    against a 1e-4 bar."""
    c = cases.make_case(5)
    w = _band(c, 7.5, 8.5, 1.9, 2.1)
    s = _setup(c)
    p, _, info = s.solve(mode="fp64", rtol=1e-13)
    assert info.status == 0
    # the adjoint source is a volume band: ||A|| ||mu|| / ||w|| is of the order of
    # the condition number, so the attainable relative residual is ~3e-11 in
    # FP64 (~1e-10 with the FP32 inner solve)
    dphi, dalpha, _, ainfo = s.adjoint(p, torch.as_tensor(w), mode="fp64", rtol=1e-10)
    assert ainfo.status == 0
    dphi, dalpha = dphi.cpu().numpy(), dalpha.cpu().numpy()
    wt = torch.as_tensor(w).cuda()
    alpha0 = torch.as_tensor(c.alpha).cuda()
    phi0 = torch.as_tensor(c.phi).cuda()

    def L(alpha, phi):
        s.assemble(alpha, phi, c.rho_w, c.rho_a, c.g, c.ref_cell)
        pp, _, inf = s.solve(mode="fp64", rtol=1e-14, p0=p, max_refine=5, raise_on_error=False)
        return float((wt * pp).sum())

    rng = np.random.default_rng(1005)
    band_cells = np.nonzero(w)[0]
    band_faces = np.nonzero(np.isin(c.owner, band_cells) | np.isin(c.neighbour, band_cells))[0]
    step = 100.0 * float(np.abs(c.phi).max())
    worst = 0.0
    for f in rng.choice(band_faces, 16, replace=False):
        e = torch.zeros(c.F, dtype=torch.float64, device="cuda")
        e[int(f)] = step
        fd = (L(alpha0, phi0 + e) - L(alpha0, phi0 - e)) / (2 * step)
        rel = abs(fd - dphi[f]) / max(abs(dphi[f]), 1e-3 * np.abs(dphi).max())
        worst = max(worst, rel)
        assert rel <= 1e-5, (f, fd, dphi[f], rel)
    print(f"dL/dphi vs central differences, worst relative deviation {worst:.2e}")
    worst = 0.0
    fc = oracle.faces(c)
    ifc = np.nonzero(fc.kind >= 2)[0]
    cand = np.unique(np.concatenate([c.owner[ifc], c.neighbour[ifc]]))
    h = 4e-3
    # the perturbed cell keeps its wet/dry flag
    cand = cand[(np.abs(c.alpha[cand] - 0.5) > 2 * h) & (np.abs(dalpha[cand]) >= 0.2 * np.abs(dalpha).max())]
    assert cand.size >= 4

    def central(i, step):
        e = torch.zeros(c.n, dtype=torch.float64, device="cuda")
        e[int(i)] = step
        return (L(alpha0 + e, phi0) - L(alpha0 - e, phi0)) / (2 * step)

    for i in rng.choice(cand, min(16, cand.size), replace=False):
        fd = (4.0 * central(i, h / 2) - central(i, h)) / 3.0
        rel = abs(fd - dalpha[i]) / abs(dalpha[i])
        worst = max(worst, rel)
        assert rel <= 1e-4, (i, fd, dalpha[i], rel)
    print(f"dL/dalpha vs Richardson central differences, worst relative deviation {worst:.2e}")


def test_adjoint_alpha_central_differences_eps_1e6_tank():
    """Central differences with eps = 1e-6 on 16 alpha entries of the
    deck-band loss, at the 1e-5 bar.  At this step the difference of two full
    solves is below their noise, so the change of L comes from an identity
    that holds for any fixed p0: L(alpha') = w.p0 + mu'.(b' - A' p0), with
    mu' = A'^{-1} w solved on the GPU after assembling at alpha'.  b' - A' p0
    is split into r0 = b - A p0 and its change, which the exported face and
    cell coefficients give to rounding (it is nonzero only around the
    perturbed cell), so the difference quotient carries the adjoint solves'
    relative error instead of the forward solves' absolute noise."""
    c = cases.make_case(5)
    w = _band(c, 7.5, 8.5, 1.9, 2.1)
    s = _setup(c)
    p, _, info = s.solve(mode="fp64", rtol=1e-13)
    assert info.status == 0
    wt = torch.as_tensor(w).cuda()
    _, dalpha, _, ainfo = s.adjoint(p, wt, mode="fp64", rtol=1e-10)
    assert ainfo.status == 0
    dalpha = dalpha.cpu().numpy()
    ex0 = {k: v.cpu().numpy() for k, v in s.export_system().items()}
    p0 = p.cpu().numpy()
    own, nb = c.owner, c.neighbour

    def apply(diag, gamma, x):  # face-form A x on the host, fixed order
        y = diag * x
        y -= np.bincount(own, weights=gamma * x[nb], minlength=c.n)
        y -= np.bincount(nb, weights=gamma * x[own], minlength=c.n)
        return y

    r0 = ex0["b"] - apply(ex0["diag"], ex0["gamma"], p0)
    alpha0 = torch.as_tensor(c.alpha).cuda()
    phi0 = torch.as_tensor(c.phi).cuda()

    def side(alpha):
        s.assemble(alpha, phi0, c.rho_w, c.rho_a, c.g, c.ref_cell)
        ex = {k: v.cpu().numpy() for k, v in s.export_system().items()}
        dr = (ex["b"] - ex0["b"]) - apply(ex["diag"] - ex0["diag"], ex["gamma"] - ex0["gamma"], p0)
        _, _, mu, inf = s.adjoint(p, wt, mode="fp64", rtol=1e-10)
        assert inf.status == 0
        return mu.cpu().numpy(), dr

    fc = oracle.faces(c)
    ifc = np.nonzero(fc.kind >= 2)[0]
    cand = np.unique(np.concatenate([c.owner[ifc], c.neighbour[ifc]]))
    cand = cand[(np.abs(c.alpha[cand] - 0.5) > 1e-3) & (w[cand] > 0)]
    rng = np.random.default_rng(2005)
    eps = 1e-6
    worst = 0.0
    for i in rng.choice(cand, min(16, cand.size), replace=False):
        e = torch.zeros(c.n, dtype=torch.float64, device="cuda")
        e[int(i)] = eps
        mu_p, dr_p = side(alpha0 + e)
        mu_m, dr_m = side(alpha0 - e)
        dL = (mu_p - mu_m) @ r0 + mu_p @ dr_p - mu_m @ dr_m
        fd = dL / (2 * eps)
        rel = abs(fd - dalpha[i]) / max(abs(dalpha[i]), 1e-3 * np.abs(dalpha).max())
        worst = max(worst, rel)
        assert rel <= 1e-5, (i, fd, dalpha[i], rel)
    print(f"dL/dalpha vs eps=1e-6 central differences, worst relative deviation {worst:.2e}")
