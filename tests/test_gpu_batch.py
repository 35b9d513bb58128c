"""Batched solve of many tanks of uneven size in one persistent launch
(per-tank CG scalars and stopping tests), against the CPU oracle tank by
tank, plus capture and replay in a CUDA graph."""
import numpy as np
import pytest
import torch

import cases
import oracle

pytestmark = pytest.mark.gpu


def _g():
    import paper_1804_01130_gb300 as g
    return g


def _tanks():
    specs = [(24, 12, 0.05, 1), (40, 20, 0.12, 2), (16, 8, 0.1, 1), (64, 16, 0.08, 3), (33, 17, 0.15, 2),
             (8, 40, 0.02, 1)]
    return [cases.box_case(nx, ny, 1, seed=100 + k, ka=ka, nwaves=nw) for k, (nx, ny, ka, nw) in enumerate(specs)]


def _phys(tanks):
    return [dict(rho_w=t.rho_w, rho_a=t.rho_a, g=t.g, ref_cell=t.ref_cell, ref_value=t.ref_value) for t in tanks]


def _cat(tanks, attr):
    return torch.as_tensor(np.concatenate([getattr(t, attr) for t in tanks]))


def test_batched_assembly_matches_oracle_per_tank():
    tanks = _tanks()
    b = _g().GFMBatch(tanks)
    b.assemble(_cat(tanks, "alpha"), _cat(tanks, "phi"), _phys(tanks))
    ex = {k: v.cpu().numpy() for k, v in b.export_system().items()}
    c0 = f0 = 0
    for t in tanks:
        fc = oracle.faces(t)
        sy = oracle.assemble(t, fc)
        assert np.array_equal(ex["gamma"][f0:f0 + t.F], fc.gamma)
        assert np.array_equal(ex["jump"][f0:f0 + t.F], fc.jump)
        assert np.array_equal(ex["diag"][c0:c0 + t.n], sy.diag)
        assert np.array_equal(ex["b"][c0:c0 + t.n], sy.b)
        c0 += t.n
        f0 += t.F


@pytest.mark.parametrize("renumber", [0, 1])
def test_batched_solve_matches_oracle_per_tank(renumber):
    tanks = _tanks()
    b = _g().GFMBatch(tanks, renumber=renumber)
    b.assemble(_cat(tanks, "alpha"), _cat(tanks, "phi"), _phys(tanks))
    p, fcorr, infos = b.solve(rtol=1e-12, phi_corr=True)
    assert len(infos) == len(tanks)
    pn = p.cpu().numpy()
    c0 = 0
    iters = []
    for t, inf in zip(tanks, infos):
        assert inf.status == 0 and inf.rel_res_l2 <= 1e-12, inf
        p_ref, _, _, _ = oracle.solve(t, direct=True)
        seg = pn[c0:c0 + t.n]
        assert np.linalg.norm(seg - p_ref) <= 1e-6 * np.linalg.norm(p_ref)
        iters.append(inf.iters)
        c0 += t.n
    # uneven tanks need uneven iteration counts: finished tanks dropped out
    assert len(set(iters)) > 1


def test_batched_converged_tank_drops_out():
    """A tank started from its exact solution finishes at once while the
    others iterate."""
    tanks = _tanks()
    b = _g().GFMBatch(tanks)
    b.assemble(_cat(tanks, "alpha"), _cat(tanks, "phi"), _phys(tanks))
    p_ref0, _, _, _ = oracle.solve(tanks[0], direct=True)
    p0 = np.zeros(sum(t.n for t in tanks))
    p0[:tanks[0].n] = p_ref0
    p, _, infos = b.solve(rtol=1e-11, p0=torch.as_tensor(p0))
    assert infos[0].status == 0 and infos[0].iters == 0
    assert all(i.status == 0 and i.iters > 0 for i in infos[1:])


def test_batched_solve_is_bit_reproducible():
    """The device re-plans the tank->CTA table as tanks finish and serves
    residual replacements in rounds; both are decided from sums every CTA
    computes in the same order, so a repeated solve (and a re-assembly)
    gives the same bits and the same iteration counts."""
    tanks = _tanks()
    b = _g().GFMBatch(tanks)
    runs = []
    for rep in range(3):
        if rep != 1:  # re-assemble before the first and the last solve
            b.assemble(_cat(tanks, "alpha"), _cat(tanks, "phi"), _phys(tanks))
        p, _, infos = b.solve(rtol=1e-11)
        runs.append((p.clone(), [(i.iters, i.refinements) for i in infos]))
    assert len(set(it for it, _ in runs[0][1])) > 1  # tanks finished at different times
    for p, its in runs[1:]:
        assert torch.equal(p, runs[0][0])
        assert its == runs[0][1]


def test_batched_128_tanks_at_the_limit():
    """The most tanks a batch takes (128): the device re-plans the CTA table
    over tanks 0..127 (each lane of the planning warp holds four), every
    tank meets its tolerance and matches the oracle."""
    g = _g()
    tanks = [cases.box_case(6 + (k % 7), 4 + (k % 5), 1, seed=500 + k, ka=0.02 + 0.001 * k, nwaves=1 + k % 3)
             for k in range(128)]
    b = g.GFMBatch(tanks)
    b.assemble(_cat(tanks, "alpha"), _cat(tanks, "phi"), _phys(tanks))
    p, _, infos = b.solve(rtol=1e-11)
    pn = p.cpu().numpy()
    c0 = 0
    for t, inf in zip(tanks, infos):
        assert inf.status == 0 and inf.rel_res_l2 <= 1e-11, inf
        p_ref, _, _, _ = oracle.solve(t, direct=True)
        assert np.linalg.norm(pn[c0:c0 + t.n] - p_ref) <= 1e-6 * np.linalg.norm(p_ref)
        c0 += t.n
    with pytest.raises(g.GFMError):
        g.GFMBatch(tanks + tanks[:1])  # 129 tanks


def test_batched_single_tank_matches_single_mesh():
    """A batch of one tank is the single-mesh problem: same assembly bits,
    solution within the mixed tolerance of the single-mesh solve."""
    g = _g()
    t = cases.box_case(48, 24, 1, seed=77, ka=0.1, nwaves=2)
    b = g.GFMBatch([t])
    b.assemble(_cat([t], "alpha"), _cat([t], "phi"), _phys([t]))
    s = g.GFM.from_case(t, renumber=1)
    s.assemble(torch.as_tensor(t.alpha), torch.as_tensor(t.phi), t.rho_w, t.rho_a, t.g, t.ref_cell, t.ref_value)
    eb = {k: v.cpu().numpy() for k, v in b.export_system().items()}
    es = {k: v.cpu().numpy() for k, v in s.export_system().items()}
    for k in ("gamma", "jump", "diag", "b"):
        assert np.array_equal(eb[k], es[k]), k
    pb, _, infos = b.solve(rtol=1e-11)
    ps, _, info = s.solve(mode="mixed", rtol=1e-11)
    assert infos[0].status == 0 and info.status == 0
    assert float(torch.linalg.norm(pb - ps) / torch.linalg.norm(ps)) <= 1e-8


def test_batched_solve_in_cuda_graph():
    tanks = _tanks()
    g = _g()
    b = g.GFMBatch(tanks)
    alpha = _cat(tanks, "alpha").cuda()
    phi = _cat(tanks, "phi").cuda()
    phys = _phys(tanks)
    out = torch.zeros(sum(t.n for t in tanks), dtype=torch.float64, device="cuda")
    # warm up (plans the launch, sets kernel attributes) before capture
    b.assemble(alpha, phi, phys)
    ref, _, infos = b.solve(rtol=1e-11)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            b.assemble(alpha, phi, phys)
            b.solve(rtol=1e-11, info_on_device=True, out=out)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(3):
        out.zero_()
        graph.replay()
    torch.cuda.synchronize()
    recs = b.infos_from_device(b._info_dev)
    assert all(r.status == 0 for r in recs)
    assert torch.allclose(out, ref, rtol=0, atol=1e-9 * float(ref.abs().max()))


def test_batched_rejects_bad_use():
    g = _g()
    tanks = _tanks()[:2]
    b = g.GFMBatch(tanks)
    bad = _phys(tanks)
    bad[1]["ref_cell"] = -1
    with pytest.raises(g.GFMError):
        b.assemble(_cat(tanks, "alpha"), _cat(tanks, "phi"), bad)
    b.assemble(_cat(tanks, "alpha"), _cat(tanks, "phi"), _phys(tanks))
    with pytest.raises(g.GFMError) as e:
        b.solve(mode="fp64")
    assert e.value.status == g.GFM_ERR_ARG


def test_batched_autotune_tank_table():
    """The autotuner may reweight the tank->CTA table by iterations; the
    batched solve still meets every tank's tolerance and matches the oracle."""
    tanks = _tanks()
    g = _g()
    b = g.GFMBatch(tanks)
    b.assemble(_cat(tanks, "alpha"), _cat(tanks, "phi"), _phys(tanks))
    threads, per_sm, ms = b.autotune(rtol=1e-11, trials=2)
    assert ms > 0.0 and threads * per_sm <= 512
    p, _, infos = b.solve(rtol=1e-11)
    pn = p.cpu().numpy()
    c0 = 0
    for t, inf in zip(tanks, infos):
        assert inf.status == 0
        p_ref, _, _, _ = oracle.solve(t, direct=True)
        assert np.linalg.norm(pn[c0:c0 + t.n] - p_ref) <= 1e-6 * np.linalg.norm(p_ref)
        c0 += t.n
