"""gfm_piso_step: the pressure part of a time step (n_solves warm-started
pressure solves on one alpha, each with its own predicted flux, then the
corrected flux, gradient and velocity of the last) as one enqueue-only
sequence, eagerly and replayed from a CUDA graph.

- The step equals the same solves made one call at a time (full assembly
  each time, warm start by hand): bit for bit.
- A replayed graph equals the eager step, bit for bit, with new fluxes.
- Warm starts pay: after the first corrector, iterations fall.
- The last solution, its gradient and velocity match the oracle's.
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


def _fluxes(c, k, seed=0, scale=1e-2):
    """Corrector fluxes: the case's predicted flux plus shrinking seeded
    changes (the SIMPLE/PISO iterations converging within a step)."""
    rng = np.random.default_rng(seed)
    mesh = dict(xf=c.xf, Sf=c.Sf, spacing=(0.1, 0.1, 0.1), dims=c.dims)
    out = [c.phi.copy()]
    for j in range(1, k):
        d = cases.random_face_flux(mesh, rng, two_d=c.dims[2] == 1)
        out.append(c.phi + scale ** j * d)
    return np.stack(out)


def _phys(c):
    return dict(rho_w=c.rho_w, rho_a=c.rho_a, g=c.g, ref_cell=c.ref_cell, ref_value=c.ref_value)


def _step(s, c, phis, n_nonorth=0, mode="mixed"):
    dev = torch.device("cuda")
    k = phis.shape[0]
    p = torch.zeros(c.n, dtype=torch.float64, device=dev)
    info = torch.zeros(4 * k, dtype=torch.float64, device=dev)
    fl = torch.empty(c.F, dtype=torch.float64, device=dev)
    G = torch.empty((3, c.n), dtype=torch.float64, device=dev)
    U = torch.empty((3, c.n), dtype=torch.float64, device=dev)
    s.piso_step(torch.as_tensor(c.alpha, device=dev), torch.as_tensor(phis, device=dev), p, info,
                V=torch.as_tensor(c.V, device=dev), xf=torch.as_tensor(c.xf, device=dev), n_nonorth=n_nonorth,
                phi_corr=fl, grad=G, U=U, mode=mode, rtol=1e-10, **_phys(c))
    torch.cuda.synchronize()
    return p, fl, G, U, s.infos_of_step(info, k)


@pytest.mark.parametrize("mk", [lambda: cases.make_case(1), lambda: cases.box_case(16, 12, 6, seed=3, permute=True)])
def test_step_equals_one_call_at_a_time(mk):
    c = mk()
    phis = _fluxes(c, 4)
    g = _g()
    s = g.GFM.from_case(c)
    p, fl, _, _, infos = _step(s, c, phis)
    assert all(i.status == 0 for i in infos)
    ref = g.GFM.from_case(c)
    q = None
    for j in range(phis.shape[0]):
        ref.assemble(torch.as_tensor(c.alpha), torch.as_tensor(phis[j]), **_phys(c))
        q, fq, inf = ref.solve(mode="mixed", rtol=1e-10, p0=q, phi_corr=True)
        assert inf.iters == infos[j].iters
    assert torch.equal(p, q) and torch.equal(fl, fq)


def test_warm_started_correctors_iterate_less():
    c = cases.make_case(2)
    phis = _fluxes(c, 6, scale=1e-2)
    s = _g().GFM.from_case(c)
    _, _, _, _, infos = _step(s, c, phis)
    its = [i.iters for i in infos]
    assert all(i.status == 0 for i in infos)
    assert max(its[1:]) < its[0], its


def test_graph_replay_equals_the_eager_step():
    c = cases.box_case(40, 20, 1, seed=5, ka=0.1)
    g = _g()
    dev = torch.device("cuda")
    k = 4
    phis_a, phis_b = _fluxes(c, k, seed=1), _fluxes(c, k, seed=2)
    s = g.GFM.from_case(c)
    alpha = torch.as_tensor(c.alpha, device=dev)
    phi_buf = torch.as_tensor(phis_a, device=dev).contiguous()
    p = torch.zeros(c.n, dtype=torch.float64, device=dev)
    info = torch.zeros(4 * k, dtype=torch.float64, device=dev)
    fl = torch.empty(c.F, dtype=torch.float64, device=dev)
    V = torch.as_tensor(c.V, device=dev)
    # warm-up outside the capture (launch plans, kernel attributes)
    s.piso_step(alpha, phi_buf, p, info, V=V, phi_corr=fl, rtol=1e-10, **_phys(c))
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(graph, stream=st):
            s.piso_step(alpha, phi_buf, p, info, V=V, phi_corr=fl, rtol=1e-10, **_phys(c), stream=st)
    torch.cuda.current_stream().wait_stream(st)
    for phis in (phis_b, phis_a):
        phi_buf.copy_(torch.as_tensor(phis, device=dev))
        p.zero_()
        graph.replay()
        torch.cuda.synchronize()
        got_p, got_fl = p.clone(), fl.clone()
        p2, fl2, _, _, infos = _step(g.GFM.from_case(c), c, phis)
        assert torch.equal(got_p, p2) and torch.equal(got_fl, fl2)
        assert [i.iters for i in s.infos_of_step(info, k)] == [i.iters for i in infos]


def test_last_corrector_matches_the_oracle():
    c = cases.box_case(24, 16, 1, seed=9, ka=0.12)
    phis = _fluxes(c, 3)
    p, fl, G, U, infos = _step(_g().GFM.from_case(c), c, phis)
    p_ref, fc, _, _ = oracle.solve(c, phi=phis[-1], direct=True)
    pn = p.cpu().numpy()
    assert np.linalg.norm(pn - p_ref) <= 1e-6 * np.linalg.norm(p_ref)
    fl_ref = oracle.corrected_flux(c, fc, pn, phi=phis[-1])
    assert np.max(np.abs(fl.cpu().numpy() - fl_ref)) <= 1e-9 * np.max(np.abs(fc.gamma * fc.jump))
    G_ref = oracle.gradient(c, pn)
    assert np.max(np.abs(G.cpu().numpy() - G_ref)) <= 1e-9 * np.max(np.abs(G_ref)) + 1e-9
    U_ref = oracle.reconstruct(c, fl.cpu().numpy())
    assert np.max(np.abs(U.cpu().numpy() - U_ref)) <= 1e-12 * np.max(np.abs(U_ref)) + 1e-15


def test_step_with_non_orthogonal_correctors():
    m = cases.wavy_mesh(32, 16)
    dy = 1.0 / 16
    alpha = np.clip((0.45 - m["C"][1]) / dy + 0.5, 0.0, 1.0)
    phi = cases.random_face_flux(m, np.random.default_rng(4), two_d=True)
    c = cases._case_from(m, alpha, phi, "wavy", (0, 15, 0))
    phis = np.stack([c.phi, c.phi * 1.01])
    s = _g().GFM.from_case(c)
    p, _, _, _, infos = _step(s, c, phis, n_nonorth=4, mode="fp64")
    assert all(i.status == 0 for i in infos)
    # the oracle's loop on the last flux, from its own start
    p_ref, _, _, _ = oracle.solve_nonorth(c, 4, phi=phis[-1], direct=True)
    assert np.linalg.norm(p.cpu().numpy() - p_ref) <= 1e-6 * np.linalg.norm(p_ref)


def test_step_argument_errors():
    g = _g()
    c = cases.box_case(8, 6, 1, seed=1)
    s = g.GFM.from_case(c)
    dev = torch.device("cuda")
    p = torch.zeros(c.n, dtype=torch.float64, device=dev)
    info = torch.zeros(4, dtype=torch.float64, device=dev)
    with pytest.raises(g.GFMError):  # grad needs V
        s.piso_step(torch.as_tensor(c.alpha, device=dev), torch.as_tensor(c.phi, device=dev)[None], p, info,
                    grad=torch.empty((3, c.n), dtype=torch.float64, device=dev), **_phys(c))
