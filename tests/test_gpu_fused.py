"""The fused form of the mixed-precision solve (one operator pass and one
grid all-reduce per FP32 iteration) against the CPU FP64 oracle, through
the C ABI.

The fused form runs the same preconditioned CG recurrences as the two-pass
form in another arrangement (the update of one step folded into the next
operator pass, r.u of the next step expanded from q.D q, t.D q and t.D t),
so the bars are the mixed-mode ones: p_d within relative L2 1e-6 of the
oracle and the true residual at the requested tolerance.  Cases span
several slices with ragged tails, 2D and 3D, permuted caller order, cached
and streamed tables, with and without the coarse space, and warm starts.
"""
import numpy as np
import pytest
import torch

import cases
import oracle

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6


def _g():
    import paper_1804_01130_gb300 as g
    return g


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _setup(case, renumber=1, form=2, stream=False, coarse=8):
    s = _g().GFM.from_case(case, renumber=renumber)
    s.set_coarse(coarse)
    s.set_table(compact=False, force_stream=stream)
    s.set_tuning(form=form)
    s.assemble(torch.as_tensor(case.alpha), torch.as_tensor(case.phi), case.rho_w, case.rho_a, case.g, case.ref_cell,
               case.ref_value)
    return s


CASES = {
    "tank_8x4": lambda: cases.box_case(8, 4, 1, seed=3, ka=0.15),
    "config1_64x32": lambda: cases.make_case(1),
    "tank_37x19_ragged": lambda: cases.box_case(37, 19, 1, seed=8, nwaves=2),
    "box_12x10x5_perm": lambda: cases.box_case(12, 10, 5, seed=4, permute=True, alpha_noise=0.1),
    "column_1x40": lambda: cases.column_case(ny=40, level=0.5173),
    "tank_300x90": lambda: cases.box_case(300, 90, 1, seed=11, nwaves=3),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("stream", [False, True])
@pytest.mark.parametrize("coarse", [8, 0])
def test_fused_solve_matches_oracle(name, stream, coarse):
    c = CASES[name]()
    p_ref, fc, sy, _ = oracle.solve(c, direct=c.n <= 2048, rtol=1e-14)
    s = _setup(c, stream=stream, coarse=coarse)
    assert s.iteration_form() == 2
    p, _, info = s.solve(mode="mixed", rtol=1e-12)
    assert info.status == 0, info
    assert info.rel_res_l2 <= 1e-12
    pn = p.cpu().numpy()
    assert _rel(pn, p_ref) <= MIXED_TOL
    # the true residual through the oracle's own matrix
    r = sy.b - oracle.spmv(sy, pn)
    assert np.linalg.norm(r) / np.linalg.norm(sy.b) <= 1.05e-12


@pytest.mark.parametrize("name", ["config1_64x32", "box_12x10x5_perm", "tank_300x90"])
def test_fused_and_two_pass_take_about_the_same_iterations(name):
    c = CASES[name]()
    p1, _, i1 = _setup(c, form=1).solve(mode="mixed", rtol=1e-10)
    p2, _, i2 = _setup(c, form=2).solve(mode="mixed", rtol=1e-10)
    assert i1.status == 0 and i2.status == 0
    # the same recurrences, rounded differently
    assert abs(i2.iters - i1.iters) <= max(5, 0.05 * i1.iters), (i1, i2)
    assert _rel(p2.cpu().numpy(), p1.cpu().numpy()) <= 1e-7


def test_fused_is_bit_reproducible_and_warm_starts():
    c = CASES["tank_300x90"]()
    s = _setup(c)
    p, _, info = s.solve(mode="mixed", rtol=1e-10)
    p = p.clone()
    p_again, _, info_again = s.solve(mode="mixed", rtol=1e-10)
    assert torch.equal(p, p_again) and info.iters == info_again.iters
    # warm start from the solution of a nearby system converges in fewer iterations
    p_ref, _, _, _ = oracle.solve(c, direct=False, rtol=1e-14)
    x0 = torch.as_tensor(p_ref * (1.0 + 1e-6))
    pw, _, iw = s.solve(mode="mixed", rtol=1e-10, p0=x0)
    assert iw.status == 0 and iw.iters < info.iters
    assert _rel(pw.cpu().numpy(), p_ref) <= MIXED_TOL


def test_fused_form_rejected_on_a_batch_and_validated():
    g = _g()
    b = g.GFMBatch(cases.batch_cases(2), renumber=1)
    with pytest.raises(g.GFMError):
        b.set_tuning(form=2)
    s = _setup(CASES["tank_8x4"](), form=1)
    with pytest.raises(g.GFMError):
        s.set_tuning(form=3)
    assert s.iteration_form() == 1


def _adjoint_rhs(c, full_width=False):
    """dL/dp: cell volumes in a band across the free surface (in 2D limited
    in x unless full_width)."""
    band = np.abs(c.C[1] - 0.5) < 0.15
    if c.dims[2] == 1 and not full_width:
        band &= (c.C[0] >= 0.5) & (c.C[0] <= 1.5)
    return np.where(band, c.V, 0.0)


@pytest.mark.parametrize("name", ["config1_64x32", "box_12x10x5_perm"])
def test_fused_adjoint_matches_oracle(name):
    """The adjoint solve (gfm_solve_adjoint) runs the same persistent solver:
    in the fused form it meets the mixed adjoint bars of the two-pass form."""
    c = CASES[name]()
    w = _adjoint_rhs(c)
    dphi_ref, dalpha_ref, mu_ref, _ = oracle.adjoint(c, w, direct=c.n <= 2048, rtol=1e-14)
    s = _setup(c)
    p, _, _ = s.solve(mode="fp64", rtol=1e-13)
    dphi, dalpha, mu, info = s.adjoint(p, torch.as_tensor(w), mode="mixed", rtol=1e-12)
    assert info.status == 0
    assert np.max(np.abs(mu.cpu().numpy() - mu_ref)) <= 1e-7 * np.abs(mu_ref).max()
    for got, ref in ((dphi, dphi_ref), (dalpha, dalpha_ref)):
        assert np.max(np.abs(got.cpu().numpy() - ref)) <= 1e-5 * np.abs(ref).max()


def test_fused_form_ends_cleanly_where_fp32_stalls():
    """A right-hand side on which FP32 inner iterations stall near 1e-12 (the
    full-width band on the 64x32 tank): both forms stop at a residual near the
    request, converged or GFM_ERR_NOT_CONVERGED, and never diverge.  The fused
    form restarts its direction on the way; a restart that kept stale step
    data once made it blow up here."""
    g = _g()
    c = CASES["config1_64x32"]()
    w = torch.as_tensor(_adjoint_rhs(c, full_width=True))
    _, _, mu_ref, _ = oracle.adjoint(c, w.numpy(), direct=True)
    for form in (1, 2):
        s = _setup(c, form=form)
        p, _, _ = s.solve(mode="fp64", rtol=1e-13)
        _, _, mu, info = s.adjoint(p, w, mode="mixed", rtol=1e-12, raise_on_error=False)
        assert info.status in (0, g.GFM_ERR_NOT_CONVERGED), (form, info)
        assert info.rel_res_l2 <= 1e-11, (form, info)
        assert np.max(np.abs(mu.cpu().numpy() - mu_ref)) <= 1e-7 * np.abs(mu_ref).max()


def test_fused_autograd_backward():
    g = _g()
    c = CASES["config1_64x32"]()
    s = g.GFM.from_case(c)
    s.set_tuning(form=2)
    alpha = torch.as_tensor(c.alpha).cuda().requires_grad_(True)
    phi = torch.as_tensor(c.phi).cuda().requires_grad_(True)
    w = torch.as_tensor(_adjoint_rhs(c)).cuda()
    phys = dict(rho_w=c.rho_w, rho_a=c.rho_a, g=c.g, ref_cell=c.ref_cell)
    p = g.GFMSolve.apply(alpha, phi, s, phys, dict(mode="mixed", rtol=1e-11))
    (w * p).sum().backward()
    dphi_ref, dalpha_ref, _, _ = oracle.adjoint(c, w.cpu().numpy(), direct=True)
    assert np.max(np.abs(phi.grad.cpu().numpy() - dphi_ref)) <= 1e-5 * np.abs(dphi_ref).max()
    assert np.max(np.abs(alpha.grad.cpu().numpy() - dalpha_ref)) <= 1e-5 * np.abs(dalpha_ref).max()


def test_fused_time_step_equals_one_call_at_a_time():
    """gfm_piso_step in the fused form: warm-started correctors, bit for bit
    the same solves made one call at a time in the same form."""
    c = CASES["tank_300x90"]()
    dev = torch.device("cuda")
    rng = np.random.default_rng(4)
    mesh = dict(xf=c.xf, Sf=c.Sf, spacing=(0.1, 0.1, 0.1), dims=c.dims)
    phis = np.stack([c.phi] + [c.phi + 1e-2 ** j * cases.random_face_flux(mesh, rng, two_d=True) for j in (1, 2, 3)])
    phys = dict(rho_w=c.rho_w, rho_a=c.rho_a, g=c.g, ref_cell=c.ref_cell, ref_value=c.ref_value)
    s = _g().GFM.from_case(c)
    s.set_tuning(form=2)
    k = phis.shape[0]
    p = torch.zeros(c.n, dtype=torch.float64, device=dev)
    info = torch.zeros(4 * k, dtype=torch.float64, device=dev)
    s.piso_step(torch.as_tensor(c.alpha, device=dev), torch.as_tensor(phis, device=dev), p, info,
                V=torch.as_tensor(c.V, device=dev), rtol=1e-10, **phys)
    torch.cuda.synchronize()
    infos = s.infos_of_step(info, k)
    assert all(i.status == 0 for i in infos)
    ref = _g().GFM.from_case(c)
    ref.set_tuning(form=2)
    q = None
    for j in range(k):
        ref.assemble(torch.as_tensor(c.alpha), torch.as_tensor(phis[j]), **phys)
        q, _, inf = ref.solve(mode="mixed", rtol=1e-10, p0=q)
        assert inf.iters == infos[j].iters
    assert torch.equal(p, q)
    assert max(i.iters for i in infos[1:]) < infos[0].iters
