"""GPU edge cases and error paths of the C ABI (no GPU fault is provoked:
every failure is a host-side argument check or a bounded device wait)."""
import ctypes

import numpy as np
import pytest
import torch

import cases
import oracle

pytestmark = pytest.mark.gpu


def _g():
    import paper_1804_01130_gb300 as g
    return g


def _setup(c, renumber=1):
    s = _g().GFM.from_case(c, renumber=renumber)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    return s


def test_two_cells_one_face():
    mesh = cases.structured_mesh(1, 2, 1, 0.1, 0.2, 0.1)
    c = cases.Case("two", 2, 1, mesh["owner"], mesh["neighbour"], mesh["Sf"], mesh["C"], mesh["V"], mesh["xf"],
                   alpha=np.array([0.8, 0.1]), phi=np.array([1e-3]), ref_cell=1, dims=(1, 2, 1))
    p_ref, _, _, _ = oracle.solve(c, direct=True)
    for mode in ("fp64", "mixed"):
        p, _, info = _setup(c).solve(mode=mode, rtol=1e-13)
        assert info.status == 0
        assert np.allclose(p.cpu().numpy(), p_ref, rtol=1e-9, atol=1e-9 * np.abs(p_ref).max())


@pytest.mark.parametrize("n", [31, 32, 33, 65])
def test_slice_boundaries(n):
    c = cases.column_case(ny=n, level=0.37)
    p_ref, _, _, _ = oracle.solve(c, direct=True)
    p, _, info = _setup(c).solve(mode="mixed", rtol=1e-13)
    assert info.status == 0
    assert np.linalg.norm(p.cpu().numpy() - p_ref) <= 1e-6 * np.linalg.norm(p_ref)


def test_alpha_tie_and_single_phase():
    c = cases.column_case(ny=8, level=0.43)
    j = np.argsort(c.C[1])
    c.alpha = np.where(c.C[1] < 0.4, 1.0, 0.0)
    c.alpha[j[3]] = 0.5
    ex = {k: v.cpu().numpy() for k, v in _setup(c).export_system().items()}
    fc = oracle.faces(c)
    assert np.array_equal(ex["lambda"], fc.lam) and np.array_equal(ex["gamma"], fc.gamma)
    c2 = cases.box_case(16, 8, 1)
    c2.alpha = np.ones(c2.n)
    p_ref, _, _, _ = oracle.solve(c2, direct=True)
    p, _, info = _setup(c2).solve(mode="fp64", rtol=1e-13)
    assert np.linalg.norm(p.cpu().numpy() - p_ref) <= 1e-9 * np.linalg.norm(p_ref)


def test_unpinned_consistent_system():
    g = _g()
    c = cases.box_case(16, 8, 1)
    s = g.GFM.from_case(c)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), ref_cell=-1)
    p, _, info = s.solve(mode="fp64", rtol=1e-11)
    assert info.status == 0
    p_ref, _, _, _ = oracle.solve(c, direct=True)
    d = p.cpu().numpy() - p_ref
    # the unpinned solution differs from the pinned one by a constant only
    assert np.ptp(d) <= 1e-7 * np.abs(p_ref).max()
    assert info.rel_res_l2 <= 1e-11


def test_argument_errors():
    g = _g()
    c = cases.box_case(8, 4, 1)
    s = g.GFM.from_case(c)
    with pytest.raises(g.GFMError) as e:
        s.solve()
    assert e.value.status == g.GFM_ERR_STATE
    with pytest.raises(g.GFMError) as e:
        s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), rho_w=1.0, rho_a=2.0)
    assert e.value.status == g.GFM_ERR_ARG
    with pytest.raises(g.GFMError) as e:
        s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), ref_cell=c.n)
    assert e.value.status == g.GFM_ERR_ARG
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi))
    with pytest.raises(g.GFMError) as e:
        s.solve(rtol=0.0)
    assert e.value.status == g.GFM_ERR_ARG
    with pytest.raises(g.GFMError) as e:
        s.set_tuning(threads=100)
    assert e.value.status == g.GFM_ERR_ARG
    with pytest.raises(g.GFMError) as e:
        s.set_tuning(threads=1024)
    assert e.value.status == g.GFM_ERR_ARG
    with pytest.raises(g.GFMError) as e:
        s.set_coarse(9)
    assert e.value.status == g.GFM_ERR_ARG
    # bad mesh: owner >= neighbour
    with pytest.raises(g.GFMError) as e:
        g.GFM(c.neighbour, c.owner, c.Sf, c.C)
    assert e.value.status == g.GFM_ERR_ARG
    # index out of range
    bad = c.neighbour.copy()
    bad[0] = c.n + 5
    with pytest.raises(g.GFMError) as e:
        g.GFM(c.owner, bad, c.Sf, c.C)
    assert e.value.status == g.GFM_ERR_ARG


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_not_converged_reports_info(mode):
    c = cases.make_case(1)
    s = _setup(c)
    p, _, info = s.solve(mode=mode, rtol=1e-12, max_iters=3, raise_on_error=False)
    g = _g()
    assert info.status == g.GFM_ERR_NOT_CONVERGED
    assert info.iters <= 3 + 1
    assert np.all(np.isfinite(p.cpu().numpy()))
    assert info.rel_res_l2 > 1e-12


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_barrier_timeout_is_reported_not_hung(mode):
    """A wait budget far below one barrier round trip makes a wait run out:
    the kernel records GFM_ERR_TIMEOUT and every CTA returns; the context
    stays usable for the next solve."""
    c = cases.box_case(64, 32, 1)
    s = _setup(c)
    p, _, info = s.solve(mode=mode, rtol=1e-12, timeout_ms=1e-6, raise_on_error=False)
    assert info.status == _g().GFM_ERR_TIMEOUT
    p, _, info = s.solve(mode=mode, rtol=1e-12)
    assert info.status == 0


def test_info_on_device_and_warm_start():
    c = cases.make_case(1)
    s = _setup(c)
    p, _, dinfo = s.solve(mode="mixed", rtol=1e-11, info_on_device=True)
    torch.cuda.synchronize()
    info = _g().GFM.info_from_device(dinfo)
    assert info.status == 0 and info.rel_res_l2 <= 1e-11
    p2, _, info2 = s.solve(mode="fp64", rtol=1e-11, p0=p)
    assert info2.status == 0
    assert info2.iters <= 2


def test_host_buffer_entry_point():
    c = cases.make_case(1)
    s = _g().GFM.from_case(c)
    a = torch.as_tensor(c.alpha).pin_memory()
    f = torch.as_tensor(c.phi).pin_memory()
    out = torch.zeros(c.n, dtype=torch.float64).pin_memory()
    info = s.solve_host(a, f, out, mode="mixed", rtol=1e-12, ref_cell=c.ref_cell)
    assert info.status == 0
    p_ref, _, _, _ = oracle.solve(c, direct=False, rtol=1e-14)
    assert np.linalg.norm(out.numpy() - p_ref) <= 1e-6 * np.linalg.norm(p_ref)


def test_tuning_shapes_agree():
    c = cases.box_case(40, 20, 1, seed=2)
    s = _setup(c)
    ref, _, _ = s.solve(mode="mixed", rtol=1e-12)
    for threads, per in [(256, 2), (512, 1), (128, 4), (64, 8)]:
        s.set_tuning(threads, per)
        p, _, info = s.solve(mode="mixed", rtol=1e-12)
        assert info.status == 0
        assert np.linalg.norm((p - ref).cpu().numpy()) <= 1e-7 * np.linalg.norm(ref.cpu().numpy())


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_coarse_space_regions_and_speedup(mode):
    """The two-level preconditioner finds one water and one air region on
    the tank, cuts the iteration count, and changes nothing in the answer."""
    c = cases.make_case(1)
    p_ref, _, _, _ = oracle.solve(c, direct=True)
    s = _setup(c)
    k, nreg, sizes = s.coarse_info()
    wet = int((c.alpha >= 0.5).sum())
    assert k == 2 and nreg == 2 and sorted(sizes) == sorted([wet, c.n - wet])
    p1, _, i1 = s.solve(mode=mode, rtol=1e-12)
    s.set_coarse(0)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell)
    assert s.coarse_info()[0] == 0
    p0, _, i0 = s.solve(mode=mode, rtol=1e-12)
    assert i1.status == 0 and i0.status == 0
    assert i1.iters < i0.iters
    for p in (p0, p1):
        assert np.linalg.norm(p.cpu().numpy() - p_ref) <= 1e-9 * np.linalg.norm(p_ref)


def test_coarse_space_many_regions_and_unpinned():
    """Floating droplets and bubbles give several regions; the kept ones are
    the largest; an unpinned system falls back to Jacobi."""
    c = cases.box_case(48, 32, 1, seed=5)
    rng = np.random.default_rng(2)
    a = c.alpha.copy()
    i = np.arange(c.n) % 48
    j = np.arange(c.n) // 48
    for (ci, cj, r, val) in [(10, 26, 3, 1.0), (30, 28, 2, 1.0), (20, 6, 3, 0.0), (40, 5, 2, 0.0)]:
        a[(i - ci) ** 2 + (j - cj) ** 2 <= r * r] = val
    c.alpha = a
    p_ref, _, _, _ = oracle.solve(c, direct=False, rtol=1e-14)
    s = _g().GFM.from_case(c)
    s.set_coarse(8, 4)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell)
    k, nreg, sizes = s.coarse_info()
    assert k == nreg and k >= 5
    assert sizes == sorted(sizes, reverse=True)
    for mode in ("fp64", "mixed"):
        p, _, info = s.solve(mode=mode, rtol=1e-12)
        assert info.status == 0
        assert np.linalg.norm(p.cpu().numpy() - p_ref) <= 1e-7 * np.linalg.norm(p_ref)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, -1)
    assert s.coarse_info()[0] == 0
    p, _, info = s.solve(mode="fp64", rtol=1e-11)
    assert info.status == 0


def test_profiling_leaves_no_stale_error():
    """Reading the profile before any solve, then destroying the handle, must
    not poison the next handle's launches."""
    c = cases.box_case(16, 8, 1)
    s = _setup(c)
    s.set_profiling(True)
    s.profile()
    s.close()
    s2 = _setup(c, renumber=2)
    p, _, info = s2.solve(mode="mixed", rtol=1e-11)
    assert info.status == 0


def test_reassembly_and_solve_are_bit_reproducible():
    """Assembly (with the coarse regions, their cross-face list and E) and
    both solves give the same bits at every repetition: no result depends on
    the order in which atomics or CTAs happen to run."""
    c = cases.make_case(2)
    g = _g()
    s = g.GFM.from_case(c, renumber=1)
    alpha, phi = torch.as_tensor(c.alpha).cuda(), torch.as_tensor(c.phi).cuda()
    first = {}
    for rep in range(6):
        s.assemble(alpha, phi, c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
        for mode in ("mixed", "fp64"):
            p, _, info = s.solve(mode=mode, rtol=1e-10)
            key = (mode, info.iters, info.refinements)
            if mode not in first:
                first[mode] = (key, p.clone())
            else:
                assert key == first[mode][0], (rep, key, first[mode][0])
                assert torch.equal(p, first[mode][1]), (rep, mode)


def test_autotune_keeps_a_valid_shape_and_the_solution():
    g = _g()
    c = cases.make_case(1)
    s = g.GFM.from_case(c)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    threads, per_sm, ms = s.autotune(mode="mixed", rtol=1e-12, trials=2)
    assert (threads, per_sm) in {(512, 1), (256, 2), (128, 4), (384, 1), (256, 1)}
    assert ms > 0.0
    p_ref, _, _, _ = oracle.solve(c, direct=True, rtol=1e-14)
    p, _, info = s.solve(mode="mixed", rtol=1e-12)
    assert info.status == 0
    assert np.linalg.norm(p.cpu().numpy() - p_ref) <= 1e-6 * np.linalg.norm(p_ref)
    with pytest.raises(g.GFMError):
        g.GFM.from_case(c).autotune()  # before assembly
